"""Mutation check of the oracle's pins (CPU only).

Plausible mistakes are planted in copies of the oracle's C source (never in
the oracle itself); each mutant is compiled and run through a compact set of
the pins (symbolic terminating series, exact plane-wave shift, dense brute
force, constant state, closed-form nodes). Every mutant must fail at least
one pin, and the unmutated source must pass all of them.
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
from tests.test_oracle_pins import _poly_case, plane_wave_eigvec

SRC = os.path.join(os.path.dirname(oracle.__file__), "stp_oracle.c")

MUTANTS = {
    "operator sign": ("pn[n * M + r] -= acc;", "pn[n * M + r] += acc;"),
    "lambda/mu swapped": ("const double lam = rho * (cp * cp - 2.0 * cs * cs);\n  const double mu = rho * cs * cs;",
                          "const double mu = rho * (cp * cp - 2.0 * cs * cs);\n  const double lam = rho * cs * cs;"),
    "factorial off by one": ("c = c * dt / (double)(k + 2);", "c = c * dt / (double)(k + 1);"),
    "one Taylor term missing": ("for (int k = 0; k + 1 < K; ++k) {", "for (int k = 0; k + 2 < K; ++k) {"),
    "D transposed": ("acc += D[i * N + l] * p[", "acc += D[l * N + i] * p["),
    "face sides swapped": ("const double* phi = side ? phi1 : phi0;", "const double* phi = side ? phi0 : phi1;"),
    "missing 1/h": ("g[NODE(z, y, x) * M + s] = acc / h;", "g[NODE(z, y, x) * M + s] = acc;"),
    "shear coefficient": ("if (d == j) B[r][i] += -mu;", "if (d == j) B[r][i] += -lam;"),
    "velocity coefficient": ("B[i][sig[i][d]] = -1.0 / rho;", "B[i][sig[i][d]] = -rho;"),
    "y-face in-plane order": ("else if (d == 1) { z = a; y = i; x = b; }", "else if (d == 1) { z = b; y = i; x = a; }"),
    "average misses q": ("memcpy(avg, q, sizeof(double) * n3 * M);", "memset(avg, 0, sizeof(double) * n3 * M);"),
    "nodes on [-1,1]": ("xi[i] = 0.5 * (t + 1.0);", "xi[i] = t;"),
}


def build_variant(tmp_path, name, src_text):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(c),
                    "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_stp.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_double] + [ctypes.c_void_p] * 5
    lib.oracle_stp.restype = ctypes.c_int
    lib.oracle_gl_nodes.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.oracle_gl_nodes.restype = ctypes.c_int
    return lib


def run(lib, q, params, h, dt):
    q = np.ascontiguousarray(q)
    params = np.ascontiguousarray(params)
    E, N = q.shape[0], q.shape[1]
    avg = np.empty_like(q)
    faces = np.empty((E, 6, N, N, 9))
    rc = lib.oracle_stp(N, N + 1, E, h, dt, q.ctypes.data, params.ctypes.data, avg.ctypes.data,
                        faces.ctypes.data, None)
    assert rc == 0
    return avg, faces


@pytest.fixture(scope="module")
def cases():
    out = {}
    # symbolic terminating series, N = 3, lambda != mu
    h, dt = 0.5, 0.03
    q, params, avg_x, faces_x = _poly_case(3, 2.0, 3.0, 1.0, h, dt, [(0.0, 0.0, 0.0), (0.5, -1.0, 1.5)], 3)
    out["poly"] = (q, params, h, dt, avg_x, faces_x)
    # exact plane-wave shift, P along x and S along y (polarised z), N = 3
    waves = []
    for axis, pol in ((0, 0), (1, 2)):
        rho, cp, cs, N = 2.3, 4.7, 2.1, 3
        hh, dtt = 0.25, 0.02
        f = np.polynomial.Polynomial([0.3, -0.7, 0.4])
        F = f.integ()
        r, c = plane_wave_eigvec(axis, pol, rho, cp, cs)
        xi, _ = ref.gl_points(N)
        coord = xi * hh
        shape = [1, 1, 1]
        shape[2 - axis] = N
        s0 = f(coord).reshape(shape)
        s1 = ((F(coord) - F(coord - c * dtt)) / (c * dtt)).reshape(shape)
        qq = np.broadcast_to(s0[..., None] * r, (N, N, N, 9))[None].copy()
        ax = np.broadcast_to(s1[..., None] * r, (N, N, N, 9))[None].copy()
        pp = np.zeros((1, N, N, N, 3))
        pp[...] = (rho, cp, cs)
        waves.append((qq, pp, hh, dtt, ax))
    out["waves"] = waves
    # dense brute force, N = 2, heterogeneous material
    rng = np.random.default_rng(5)
    N = 2
    pp = np.stack([rng.uniform(2, 3, (1, N, N, N)), rng.uniform(4, 6, (1, N, N, N)),
                   rng.uniform(1, 2, (1, N, N, N))], axis=-1)
    qq = rng.uniform(-1, 1, (1, N, N, N, 9))
    L = ref.dense_operator(N, 0.2, pp[0])
    out["dense"] = (qq, pp, 0.2, 0.004,
                    ref.dense_time_average(L, qq[0].reshape(-1), 0.004, N + 1).reshape(1, N, N, N, 9))
    return out


def pins_fail(lib, cases) -> list:
    failed = []
    q, params, h, dt, avg_x, faces_x = cases["poly"]
    avg, faces = run(lib, q, params, h, dt)
    if ref.rel_err(avg, avg_x) > 1e-12:
        failed.append("poly avg")
    if ref.rel_err(faces, faces_x) > 1e-12:
        failed.append("poly faces")
    for i, (qq, pp, hh, dtt, ax) in enumerate(cases["waves"]):
        a, _ = run(lib, qq, pp, hh, dtt)
        if ref.rel_err(a, ax) > 1e-12:
            failed.append(f"wave {i}")
    qq, pp, hh, dtt, ax = cases["dense"]
    a, _ = run(lib, qq, pp, hh, dtt)
    if ref.rel_err(a, ax) > 1e-13:
        failed.append("dense")
    xi = np.zeros(3)
    w = np.zeros(3)
    lib.oracle_gl_nodes(3, xi.ctypes.data, w.ctypes.data)
    closed = (np.array([-math.sqrt(3 / 5), 0.0, math.sqrt(3 / 5)]) + 1) / 2
    if np.abs(xi - closed).max() > 2e-16:
        failed.append("nodes")
    return failed


def test_unmutated_oracle_passes_the_compact_pins(tmp_path, cases):
    lib = build_variant(tmp_path, "original", open(SRC).read())
    assert pins_fail(lib, cases) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_planted_mistake_is_caught(tmp_path, cases, name):
    text = open(SRC).read()
    old, new = MUTANTS[name]
    assert text.count(old) == 1, f"mutation site not unique: {name}"
    lib = build_variant(tmp_path, name.replace(" ", "_").replace("/", "_"), text.replace(old, new))
    assert pins_fail(lib, cases), f"mutant '{name}' passed every pin"
