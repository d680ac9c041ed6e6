"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/stp.h declares, and its host-computed tables agree with closed forms,
a 50-digit reference and the oracle's independent construction. Argument
errors that are detected before any CUDA call are checked too. No kernel runs.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _binding.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "stp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("stp_create", "stp_predict", "stp_destroy", "stp_predict_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_has_no_oracle_dependency():
    # the product library must not link or embed the oracle
    data = open(build.LIB, "rb").read()
    assert b"oracle_stp" not in data and b"liboracle" not in data


def test_status_strings(lib):
    for s in range(0, -6, -1):
        assert stp.stp_status_string(s) != "unknown status"


@pytest.mark.parametrize("N", range(1, 13))
def test_library_tables_match_oracle_tables(lib, N):
    xi = np.zeros(N)
    D = np.zeros((N, N))
    p0 = np.zeros(N)
    p1 = np.zeros(N)
    stp.stp_reference_tables(N - 1, xi, D, p0, p1)
    xo, Do, p0o, p1o = oracle.tables(N)
    assert np.abs(xi - xo).max() <= 4e-16
    assert np.abs(D - Do).max() <= 1e-14 * max(1.0, np.abs(Do).max())
    assert np.abs(p0 - p0o).max() <= 2e-14 and np.abs(p1 - p1o).max() <= 2e-14


@pytest.mark.parametrize("N", range(2, 13))
def test_library_gauss_lobatto_tables_match_oracle_tables(lib, N):
    xi = np.zeros(N)
    D = np.zeros((N, N))
    p0 = np.zeros(N)
    p1 = np.zeros(N)
    stp.stp_reference_tables(N - 1, xi, D, p0, p1, family="gll")
    xo, Do, p0o, p1o = oracle.tables(N, "gll")
    assert np.abs(xi - xo).max() <= 4e-16
    assert np.abs(D - Do).max() <= 1e-14 * max(1.0, np.abs(Do).max())
    assert np.array_equal(p0, p0o) and np.array_equal(p1, p1o)  # unit vectors


def test_node_family_errors_before_touching_the_gpu(lib):
    with pytest.raises(stp.STPError) as ei:  # Gauss-Lobatto needs N >= 2
        stp.stp_create(0, 9, 0.1, 0.01, nodes="gll")
    assert ei.value.status == _binding.STP_ERR_UNSUPPORTED
    with pytest.raises(stp.STPError) as ei:
        stp.stp_create(3, 9, 0.1, 0.01, nodes=7)
    assert ei.value.status == _binding.STP_ERR_UNSUPPORTED
    with pytest.raises(stp.STPError):
        stp.stp_reference_tables(0, np.zeros(1), family="gll")
    assert lib.stp_get_nodes(None) == 0


@pytest.mark.parametrize("N", [3, 8, 12])
def test_library_tables_against_50_digits(lib, N):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    xi = np.zeros(N)
    D = np.zeros((N, N))
    p1 = np.zeros(N)
    stp.stp_reference_tables(N - 1, xi, D, None, p1)
    nodes = [mp.findroot(lambda x: mpmath.legendre(N, 2 * x - 1), mp.mpf(x)) for x in xi]
    for i in range(N):
        for j in range(N):
            # product-rule derivative of the j-th Lagrange polynomial at node i
            s = mp.mpf(0)
            for m in range(N):
                if m == j:
                    continue
                t = 1 / (nodes[j] - nodes[m])
                for l in range(N):
                    if l not in (j, m):
                        t *= (nodes[i] - nodes[l]) / (nodes[j] - nodes[l])
                s += t
            assert abs(D[i, j] - float(s)) <= 2e-15 * max(1.0, float(abs(s))) + 1e-15 * N * N
        lj = mpmath.fprod([(1 - nodes[l]) / (nodes[i] - nodes[l]) for l in range(N) if l != i])
        assert abs(p1[i] - float(lj)) <= 2e-15


def test_reference_tables_reject_bad_order(lib):
    with pytest.raises(stp.STPError) as ei:
        stp.stp_reference_tables(12)
    assert ei.value.status == _binding.STP_ERR_UNSUPPORTED


def test_create_rejects_before_touching_the_gpu(lib):
    for args, status in [((7, 8, 0.1, 0.01), _binding.STP_ERR_UNSUPPORTED),
                         ((12, 9, 0.1, 0.01), _binding.STP_ERR_UNSUPPORTED),
                         ((-2, 9, 0.1, 0.01), _binding.STP_ERR_UNSUPPORTED),
                         ((3, 9, 0.0, 0.01), _binding.STP_ERR_INVALID_ARG),
                         ((3, 9, 0.1, -1.0), _binding.STP_ERR_INVALID_ARG),
                         ((3, 9, math.inf, 0.01), _binding.STP_ERR_INVALID_ARG),
                         ((3, 9, 0.1, math.nan), _binding.STP_ERR_INVALID_ARG)]:
        with pytest.raises(stp.STPError) as ei:
            stp.stp_create(*args)
        assert ei.value.status == status, args


def test_predict_rejects_null_handle(lib):
    with pytest.raises(stp.STPError) as ei:
        stp.stp_predict(None, 1, 16, 16, 16, 16)
    assert ei.value.status == _binding.STP_ERR_INVALID_ARG
    stp.stp_destroy(None)  # NULL is a no-op


def test_predict_curvilinear_rejects_null_handle(lib):
    with pytest.raises(stp.STPError) as ei:
        stp.stp_predict_curvilinear(None, 1, 16, 16, 16, 16, 16)
    assert ei.value.status == _binding.STP_ERR_INVALID_ARG
    # a negative element count is rejected before the handle is used
    assert lib.stp_predict_curvilinear(None, -1, None, None, None, None, None, None) == \
        _binding.STP_ERR_INVALID_ARG


def test_batch_create_curvilinear_rejects_missing_metrics(lib):
    out = ctypes.c_void_p()
    assert lib.stp_batch_create_curvilinear(1, None, None, ctypes.byref(out)) == \
        _binding.STP_ERR_INVALID_ARG
    assert lib.stp_batch_create_curvilinear(-1, None, None, ctypes.byref(out)) == \
        _binding.STP_ERR_INVALID_ARG


def test_server_add_sim_curvilinear_rejects_null_arguments(lib):
    i = ctypes.c_int()
    assert lib.stp_server_add_sim_curvilinear(None, None, 1, None, None, None, ctypes.byref(i)) == \
        _binding.STP_ERR_INVALID_ARG


def test_static_curvilinear_batch_rejects_missing_metrics(lib):
    assert lib.stp_batch_run_static_curvilinear(1, None, None, None) == _binding.STP_ERR_INVALID_ARG
    assert lib.stp_batch_run_static_curvilinear(-1, None, None, None) == _binding.STP_ERR_INVALID_ARG


def test_predict_sources_rejects_bad_source_list(lib):
    assert lib.stp_predict_sources(None, 1, None, None, None, None, -1, None, None) == \
        _binding.STP_ERR_INVALID_ARG
    assert lib.stp_predict_sources(None, 1, None, None, None, None, 1, None, None) == \
        _binding.STP_ERR_INVALID_ARG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _binding.load()


def test_binding_precision_names_match_the_header_enum():
    text = open(os.path.join(ROOT, "include", "stp.h")).read()
    body = text[text.index("typedef enum {\n  STP_PRECISION_FP64"):text.index("} stp_precision;")]
    enum = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"STP_PRECISION_(\w+)\s*=\s*(\d+)", body)}
    assert enum == _binding.PRECISIONS


def test_set_precision_rejects_null_handle(lib):
    assert lib.stp_set_precision(None, 0) == _binding.STP_ERR_INVALID_ARG
    assert lib.stp_get_precision(None) == 0


def test_server_and_batch_entries_reject_bad_arguments_before_the_gpu(lib):
    """Every served and batched entry point checks its handle and arguments
    before any CUDA call; NULL handles are no-ops for the destroy calls."""
    bad = _binding.STP_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    assert lib.stp_server_create(1 << 20, 1, None) == bad
    assert lib.stp_server_create(0, 1, ctypes.byref(out)) == bad and not out.value
    assert lib.stp_server_create(-5, 1, ctypes.byref(out)) == bad
    assert lib.stp_server_create(1 << 20, 0, ctypes.byref(out)) == bad
    assert lib.stp_server_create(1 << 20, 9, ctypes.byref(out)) == bad
    sid, n = ctypes.c_int(), ctypes.c_int()
    steps = ctypes.c_int64()
    stats = (ctypes.c_int64 * 16)()
    assert lib.stp_server_add_sim(None, None, 1, None, None, ctypes.byref(sid)) == bad
    assert lib.stp_server_submit(None, 0) == bad
    assert lib.stp_server_progress(None, ctypes.byref(n)) == bad
    assert lib.stp_server_drain(None) == bad
    assert lib.stp_server_run_trace(None, 0, None, None, None, None) == bad
    assert lib.stp_server_read(None, 0, None, None, ctypes.byref(steps)) == bad
    assert lib.stp_server_stats(None, stats) == bad
    assert lib.stp_server_destroy(None) == _binding.STP_OK
    assert lib.stp_batch_create(1, None, ctypes.byref(out)) == bad
    assert lib.stp_batch_create(-1, None, ctypes.byref(out)) == bad
    assert lib.stp_batch_create(0, None, None) == bad
    assert lib.stp_batch_launch(None, None) == bad
    assert lib.stp_batch_info(None, None, None, None) == bad
    assert lib.stp_batch_destroy(None) == _binding.STP_OK
    sets = (ctypes.c_byte * (129 * 256))()  # contents never read: the count is checked first
    assert lib.stp_batch_run_static(129, sets, None) == bad
    assert lib.stp_batch_run_static(-1, None, None) == bad
    assert lib.stp_batch_run_static(1, None, None) == bad
    assert lib.stp_measure_fp64_peak(None, None) == bad
    # the message of the last failure names the problem
    assert lib.stp_server_create(1 << 20, 0, ctypes.byref(out)) == bad
    assert b"slots" in lib.stp_last_error()


def test_every_entry_point_is_documented_in_the_header():
    """Each declaration in include/stp.h follows a comment (its own, or the
    block that documents a group of related calls declared together)."""
    lines = open(os.path.join(ROOT, "include", "stp.h")).read().splitlines()
    decl = re.compile(r"^(stp_status|const char\*|int|void|double|int64_t) (stp_\w+)\(")
    cont = re.compile(r"^\s+\S.*[,;)]\s*$")  # continuation lines of a declaration
    undocumented = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and (not lines[j].strip() or decl.match(lines[j]) or cont.match(lines[j])):
            j -= 1
        if j < 0 or not lines[j].rstrip().endswith("*/"):
            undocumented.append(m.group(2))
    assert not undocumented, undocumented


def test_product_and_oracle_share_no_code():
    """The product (package, CUDA sources, header) never imports, includes or
    links the oracle, and the oracle never imports the product."""
    pkg = os.path.join(ROOT, "paper_2003_12787_gb300")
    for path in glob_sources(pkg) + [os.path.join(ROOT, "include", "stp.h")]:
        text = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), path
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), path
        assert "stp_oracle" not in text, path
    for name in ("__init__.py", "stp_oracle.c"):
        text = open(os.path.join(ROOT, "oracle", name)).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2003_12787_gb300", text, re.M), name
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*(stp\.h|csrc)", text), name
    assert "TEST INFRASTRUCTURE ONLY" in open(os.path.join(ROOT, "oracle", "__init__.py")).read()


def glob_sources(pkg):
    out = []
    for d, _, files in os.walk(pkg):
        out += [os.path.join(d, f) for f in files
                if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp"))]
    return out


def test_reference_tables_binding_checks_its_buffers(lib):
    """The binding refuses output buffers the library would overrun or
    misread (wrong dtype, too short, not contiguous) before calling it."""
    N = 5
    for bad in (np.zeros(N, dtype=np.float32), np.zeros(N - 1), np.zeros(2 * N)[::2]):
        with pytest.raises(ValueError):
            stp.stp_reference_tables(N - 1, bad)
    with pytest.raises(ValueError):
        stp.stp_reference_tables(N - 1, np.zeros(N), np.zeros(N * N - 1))
    xi, D = np.zeros(N), np.zeros((N, N))
    stp.stp_reference_tables(N - 1, xi, D)
    assert np.all(np.diff(xi) > 0) and np.abs(D.sum(axis=1)).max() < 1e-12  # D 1 = 0


def test_run_trace_binding_checks_its_buffers(lib):
    """A trace whose arrays have the wrong dtype or length is refused before
    the library reads them (the server handle is never touched)."""
    t = np.linspace(0.0, 1.0, 4)
    ids = np.zeros(4, dtype=np.int32)
    lat = np.zeros(4)
    for args in ((t.astype(np.float32), ids, lat), (t, ids.astype(np.int64), lat),
                 (t, ids, np.zeros(3)), (t, ids[:3], lat)):
        with pytest.raises(ValueError):
            stp.stp_server_run_trace(None, *args)
    with pytest.raises(stp.STPError):  # well-formed arrays reach the library: NULL server
        stp.stp_server_run_trace(None, t, ids, lat)


@pytest.mark.parametrize("std,lang,compiler", [("c99", "c", "gcc"), ("c11", "c", "gcc"),
                                               ("c++17", "c++", "g++")])
def test_header_stands_alone_in_c_and_cpp(tmp_path, std, lang, compiler):
    """include/stp.h needs no CUDA or torch header: it compiles on its own as
    C99, C11 and C++17 with warnings as errors."""
    import shutil
    import subprocess
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not available")
    subprocess.run([compiler, f"-std={std}", "-fsyntax-only", "-Wall", "-Wextra", "-Werror",
                    "-pedantic", "-x", lang, os.path.join(ROOT, "include", "stp.h")], check=True)


def test_plain_c_user_links_against_the_library_alone(lib, tmp_path):
    """The C example (tests/c/abi_host_predict.c) compiles with gcc and links
    against the library with no CUDA, torch or Python flags (it runs in the
    GPU tests)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    so = build.LIB
    exe = tmp_path / "abi_host_predict"
    subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host_predict.c"), "-o", str(exe),
                    "-L", os.path.dirname(so), "-l:" + os.path.basename(so),
                    "-Wl,-rpath," + os.path.dirname(so)], check=True)
    assert exe.exists()


@pytest.mark.parametrize("family,Ns", [("gl", range(1, 13)), ("gll", range(2, 13))])
def test_library_tables_have_the_symmetry_the_even_odd_kernels_use(lib, family, Ns):
    """Both node families are symmetric about 1/2, so the library's D is
    centro-antisymmetric (D[N-1-i][N-1-l] = -D[i][l]) and phi(1) mirrors
    phi(0); on such a D the even-odd split (sums and differences of mirrored
    values against the even and odd halves of D) reproduces D u."""
    rng = np.random.default_rng(7)
    for N in Ns:
        xi, D, p0, p1 = np.zeros(N), np.zeros((N, N)), np.zeros(N), np.zeros(N)
        stp.stp_reference_tables(N - 1, xi, D, p0, p1, family=family)
        scale = max(1.0, np.abs(D).max())
        assert np.abs(xi + xi[::-1] - 1.0).max() <= 2e-16, N
        assert np.abs(D[::-1, ::-1] + D).max() <= 4e-15 * scale, N
        assert np.abs(p1 - p0[::-1]).max() <= 4e-16, N
        u = rng.standard_normal(N)
        h = N // 2
        e = u[:h] + u[::-1][:h]
        o = u[:h] - u[::-1][:h]
        Dv = np.empty(N)
        for i in range(h):
            E_i = (D[i, :h] + D[i, ::-1][:h]) / 2
            O_i = (D[i, :h] - D[i, ::-1][:h]) / 2
            P = E_i @ e + (D[i, h] * u[h] if N % 2 else 0.0)
            Q = O_i @ o
            Dv[i], Dv[N - 1 - i] = P + Q, Q - P
        if N % 2:
            Dv[h] = ((D[h, :h] - D[h, ::-1][:h]) / 2) @ o
        assert np.abs(Dv - D @ u).max() <= 1e-13 * scale * np.abs(u).sum(), N
