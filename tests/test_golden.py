"""The oracle against the fixtures in tests/golden/ (CPU only).

gl_nodes_closed_form.txt holds Gauss-Legendre nodes from their closed forms
(written by tests/golden/make_golden.py with mpmath, without any node routine
of a library or of the oracle). The oracle_order*_seed*.txt files are
regression fixtures of the oracle's own outputs on small seeded cases (two
Cartesian, one curvilinear): they catch any later, unintended change of its
arithmetic.
"""
from __future__ import annotations

import importlib.util
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_values(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def generator():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLDEN, "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_nodes_match_closed_forms():
    rows = read_values("gl_nodes_closed_form.txt")
    assert [int(r[0]) for r in rows] == [1, 2, 3, 4, 5]
    for r in rows:
        N = int(r[0])
        expect = np.array([float(x) for x in r[1:]])
        xi, _ = oracle.gl_nodes(N)
        assert np.abs(xi - expect).max() <= 2e-16, N


@pytest.mark.parametrize("N,seed", [(2, 11), (3, 12)])
def test_oracle_matches_its_regression_fixture(N, seed):
    rows = read_values(f"oracle_order{N - 1}_seed{seed}.txt")
    stored = np.array([float(r[0]) for r in rows])
    text = generator().oracle_case(N, seed)
    now = np.array([float(line) for line in text.splitlines() if line and not line.startswith("#")])
    assert stored.shape == now.shape
    assert np.abs(now - stored).max() <= 1e-15 * np.abs(stored).max()


def test_curvilinear_oracle_matches_its_regression_fixture():
    rows = read_values("oracle_curvilinear_order2_seed13.txt")
    stored = np.array([float(r[0]) for r in rows])
    text = generator().oracle_curv_case(3, 13)
    now = np.array([float(line) for line in text.splitlines() if line and not line.startswith("#")])
    assert stored.shape == now.shape
    assert np.abs(now - stored).max() <= 1e-15 * np.abs(stored).max()
