"""Mutation check of the corrector oracle's pins (CPU only).

Plausible mistakes are planted in a copy of corrector_oracle.c (never in the
oracle itself), compiled beside an unchanged copy of stp_oracle.c, and run
through a compact set of the pins of test_oracle_corrector.py. Every mutant
must fail at least one pin; the unmutated source must pass all of them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import _elastic as ref
from tests import test_oracle_corrector as pins

HERE = os.path.dirname(oracle.__file__)
STP_SRC = os.path.join(HERE, "stp_oracle.c")
COR_SRC = os.path.join(HERE, "corrector_oracle.c")

MUTANTS = {
    "central flux sign": ("const double bn = sign * 0.5 *", "const double bn = -sign * 0.5 *"),
    "dissipation sign": ("(r == s ? smax : 0.0)", "(r == s ? -smax : 0.0)"),
    "jump sign": ("* (qp[s] - qm[s]);", "* (qm[s] - qp[s]);"),
    "flux without the half": ("F[r] = 0.5 * acc;", "F[r] = acc;"),
    "lift multiplies by the weight": ("phi[i] / (w[i] * h);", "phi[i] * w[i] / h;"),
    "lift on the wrong side": ("const double* phi = side ? phi1 : phi0;\n        for (int a = 0; a < N; ++a)\n          for (int b = 0; b < N; ++b) {\n            const double* qm",
                               "const double* phi = side ? phi0 : phi1;\n        for (int a = 0; a < N; ++a)\n          for (int b = 0; b < N; ++b) {\n            const double* qm"),
    "neighbour direction": ("neighbour(gx, gy, gz, e, d, side ? 1 : -1)", "neighbour(gx, gy, gz, e, d, side ? -1 : 1)"),
    "own material on both sides": ("oracle_elastic_B(d, mp[0], mp[1], mp[2], Bp);", "oracle_elastic_B(d, mm[0], mm[1], mm[2], Bp);"),
    "speed from own side only": ("fmax(fabs(mm[1]), fabs(mp[1]))", "fabs(mm[1])"),
    "y-face in-plane order": ("if (d == 1) return node_index(N, a, i, b);", "if (d == 1) return node_index(N, b, i, a);"),
    "volume term sign": ("rate[(size_t)n * M + r] -= acc;", "rate[(size_t)n * M + r] += acc;"),
    "time step missing": ("q[e * n3m + t] + dt * rate[t]", "q[e * n3m + t] + rate[t]"),
    "neighbour face index": ("const int f = 2 * d + side, fo = 2 * d + (1 - side);",
                             "const int f = 2 * d + side, fo = 2 * d + side;"),
}


class Lib:
    def __init__(self, so):
        lib = ctypes.CDLL(so)
        lib.oracle_stp_nodes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                         ctypes.c_double, ctypes.c_double] + [ctypes.c_void_p] * 5
        lib.oracle_stp_nodes.restype = ctypes.c_int
        lib.oracle_correct.argtypes = [ctypes.c_int] * 5 + [ctypes.c_double] * 2 + [ctypes.c_void_p] * 5
        lib.oracle_correct.restype = ctypes.c_int
        self.lib = lib

    def stp(self, q, params, h, dt):
        q = np.ascontiguousarray(q)
        params = np.ascontiguousarray(params)
        E, N = q.shape[0], q.shape[1]
        avg = np.empty_like(q)
        faces = np.empty((E, 6, N, N, 9))
        assert self.lib.oracle_stp_nodes(0, N, N + 1, E, h, dt, q.ctypes.data, params.ctypes.data,
                                         avg.ctypes.data, faces.ctypes.data, None) == 0
        return avg, faces

    def correct(self, q, params, avg, faces, grid, h, dt):
        arrs = [np.ascontiguousarray(a) for a in (q, params, avg, faces)]
        out = np.empty_like(arrs[0])
        N = q.shape[1]
        assert self.lib.oracle_correct(0, N, *grid, h, dt, *[a.ctypes.data for a in arrs],
                                       out.ctypes.data) == 0
        return out

    def step(self, q, params, grid, h, dt):
        avg, faces = self.stp(q, params, h, dt)
        return self.correct(q, params, avg, faces, grid, h, dt)


def build(tmp_path, name, cor_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(cor_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", STP_SRC,
                    str(c), "-o", str(so), "-lm"], check=True)
    return Lib(str(so))


@pytest.fixture(scope="module")
def cases():
    out = {}
    out["poly"] = pins._exact_poly_step(3, 2.0, 3.0, 1.0, 0.5, 0.03, seed=43)
    grid = (2, 2, 3)
    q, _ = pins.periodic_field(3, grid, 0.3, seed=71)
    out["energy"] = (q, grid)
    rng = np.random.default_rng(95)
    n = 6
    out["fv"] = (rng.uniform(-1, 1, (n, 1, 1, 1, 9)),
                 np.stack([rng.uniform(2, 3, n), rng.uniform(4, 6, n), rng.uniform(2, 3, n)],
                          axis=1).reshape(n, 1, 1, 1, 3))
    dense = []
    for N, g in ((2, (2, 1, 1)), (2, (1, 2, 1)), (2, (1, 1, 2))):
        q, params = pins.periodic_field(N, g, 0.25, seed=200 + sum(g))
        dense.append((q, params, g, pins.dense_corrector(q, params, g, 0.25, 0.004)))
    out["dense"] = dense
    return out


def failures(lib, cases):
    failed = []
    # polynomial interior element
    q, exact, grid = cases["poly"]
    o = lib.step(q, pins.uniform_params(27, 3, 2.0, 3.0, 1.0), grid, 0.5, 0.03)
    if not ref.rel_err(o[13], exact[13]) <= 1e-13:
        failed.append("polynomial")
    # energy identity
    q, grid = cases["energy"]
    E, N, h = q.shape[0], q.shape[1], 0.3
    rho, cp, cs = 2.4, 5.1, 2.2
    params = pins.uniform_params(E, N, rho, cp, cs)
    H = pins.energy_matrix(rho, cp, cs)
    _, w = ref.gl_points(N)
    fq = pins.face_values(q, N)
    rate = lib.correct(q, params, q, fq, grid, h, 1.0) - q
    W = np.einsum("i,j,k->ijk", w, w, w) * h ** 3
    dEdt = float(np.einsum("zyx,ezyxs,st,ezyxt->", W, q, H, rate))
    Wf = np.outer(w, w) * h * h
    diss = 0.0
    for e in range(E):
        for d in range(3):
            jump = fq[pins.neighbours(grid, e, d), 2 * d] - fq[e, 2 * d + 1]
            diss += float(np.einsum("ab,abs,st,abt->", Wf, jump, H, jump))
    if not abs(dEdt + 0.5 * cp * diss) <= 1e-11 * abs(0.5 * cp * diss):
        failed.append("energy")
    # first-order Rusanov with element-wise material
    q, params = cases["fv"]
    n, h, dt = q.shape[0], 0.2, 0.011
    o = lib.step(q, params, (n, 1, 1), h, dt).reshape(n, 9)
    mat = params.reshape(n, 3)
    u = q.reshape(n, 9)
    B = [-ref.coefficient_matrices(*mat[i])[0] for i in range(n)]
    fv = u.copy()
    for i in range(n):
        r, l = (i + 1) % n, (i - 1) % n
        Br, sr = 0.5 * (B[i] + B[r]), max(mat[i, 1], mat[r, 1])
        Bl, sl = 0.5 * (B[l] + B[i]), max(mat[l, 1], mat[i, 1])
        fv[i] = u[i] - dt / h * (0.5 * (Br - sr * np.eye(9)) @ (u[r] - u[i])
                                 + 0.5 * (Bl + sl * np.eye(9)) @ (u[i] - u[l]))
    if not ref.rel_err(o, fv) <= 1e-14:
        failed.append("finite volume")
    # dense brute force in each direction
    for q, params, g, dense in cases["dense"]:
        if not ref.rel_err(lib.step(q, params, g, 0.25, 0.004), dense) <= 1e-13:
            failed.append(f"dense {g}")
    return failed


def test_unmutated_source_passes_every_pin(tmp_path, cases):
    with open(COR_SRC) as f:
        lib = build(tmp_path, "clean", f.read())
    assert failures(lib, cases) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, cases, name):
    old, new = MUTANTS[name]
    with open(COR_SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site of {name!r} not unique"
    lib = build(tmp_path, "mutant", src.replace(old, new))
    assert failures(lib, cases), f"no pin caught the mutant {name!r}"
