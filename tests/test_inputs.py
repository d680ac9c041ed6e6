"""The seeded input generators (CPU): the sample points are the node family's
points, the curvilinear metric is the inverse of the map's Jacobian (checked
against central finite differences of the map itself), the state is the
plane-wave sum at the mapped positions, and the recipes are reproducible."""
from __future__ import annotations

import math

import numpy as np
import torch

from paper_2003_12787_gb300 import inputs
from tests import _elastic as ref


def test_sample_points_are_the_node_families():
    for N in range(1, 13):
        assert np.allclose(inputs.sample_points(N, "gl"), ref.gl_points(N)[0], atol=1e-15)
    for N in range(2, 13):
        assert np.allclose(inputs.sample_points(N, "gll"), ref.gll_points(N)[0], atol=1e-14)


def _mapped(X, a):
    """x(X) of the curvilinear recipe, X of shape [..., 3]."""
    tw = 2 * math.pi
    x = X.copy()
    for j in range(3):
        x[..., j] += a / tw * np.sin(tw * X[..., (j + 1) % 3]) * np.sin(tw * X[..., (j + 2) % 3])
    return x


def test_curvilinear_metric_inverts_the_map_jacobian():
    N, grid, a = 4, (3, 2, 2), 0.2
    prob = inputs.curvilinear_problem(N, grid=grid, amplitude=a)
    h, xi = prob.h, inputs.sample_points(N)
    G = prob.metric.numpy()
    Gx, Gy, _ = grid
    eps = 1e-6
    for e in range(prob.E):
        ex, ey, ez = e % Gx, (e // Gx) % Gy, e // (Gx * Gy)
        for z, y, x in [(0, 0, 0), (1, 2, 3), (3, 3, 3), (2, 0, 1)]:
            X = (np.array([ex, ey, ez]) + np.array([xi[x], xi[y], xi[z]])) * h
            # dx/dxi by central differences of the map of the reference point
            J = np.empty((3, 3))
            for m in range(3):
                d = np.zeros(3)
                d[m] = eps * h
                J[:, m] = (_mapped(X + d, a) - _mapped(X - d, a)) / (2 * eps)
            assert np.abs(G[e, z, y, x] @ J - np.eye(3)).max() <= 1e-7


def test_curvilinear_state_is_the_plane_wave_sum_at_mapped_positions():
    N, grid = 3, (2, 2, 1)
    prob = inputs.curvilinear_problem(N, grid=grid, seed_waves=77)
    k, amp, phase = inputs.wave_parameters(77)
    xi = inputs.sample_points(N)
    h = prob.h
    e, z, y, x = 3, 1, 2, 0
    ex, ey, ez = e % 2, (e // 2) % 2, e // 4
    X = (np.array([ex, ey, ez]) + np.array([xi[x], xi[y], xi[z]])) * h
    pos = _mapped(X, 0.2)
    expect = [sum(amp[w, s] * math.sin(k[w] @ pos + phase[w, s]) for w in range(len(k)))
              for s in range(9)]
    assert np.abs(prob.q[e, z, y, x].numpy() - np.array(expect)).max() <= 1e-13


def test_recipes_are_reproducible_and_cartesian_for_zero_amplitude():
    a = inputs.curvilinear_problem(5, E=9, seed_material=5, seed_waves=6)
    b = inputs.curvilinear_problem(5, E=9, seed_material=5, seed_waves=6)
    assert torch.equal(a.q, b.q) and torch.equal(a.metric, b.metric) and a.dt == b.dt
    c = inputs.curvilinear_problem(5, E=9, seed_material=5, seed_waves=6, amplitude=0.0)
    d = inputs.elastic_problem(5, E=9, seed_material=5, seed_waves=6)
    assert torch.equal(c.q, d.q) and torch.equal(c.params, d.params)
    assert torch.equal(c.metric, torch.eye(3, dtype=torch.float64).expand_as(c.metric) / c.h)
    r1, r2 = inputs.batched_sets_recipe(), inputs.batched_sets_recipe()
    assert r1 == r2 and len(r1) == 64
