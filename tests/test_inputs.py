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


def test_workloads_follow_their_stated_distributions():
    """Material, time step, plane waves, set sizes and arrivals: the ranges
    and formulas the workload descriptions state."""
    prob = inputs.small_case()
    N, E = prob.N, prob.E
    assert (N, E, prob.h, prob.grid) == (4, 512, 1.0 / 8, (8, 8, 8))
    rho, cp, cs = (prob.params[..., i].numpy() for i in range(3))
    assert rho.min() >= 2.0 and rho.max() <= 3.0 and cp.min() >= 4.0 and cp.max() <= 6.0
    assert np.abs(cs * math.sqrt(3.0) - cp).max() <= 1e-14 * cp.max()
    # the draws fill their ranges (2048 and more samples each)
    assert rho.max() - rho.min() > 0.95 and cp.max() - cp.min() > 1.9
    assert prob.dt == 0.4 * prob.h / ((2 * N - 1) * cp.max())
    k, amp, phase = inputs.wave_parameters(1002)
    assert k.shape == (4, 3) and amp.shape == (4, 9) and phase.shape == (4, 9)
    assert np.linalg.norm(k, axis=1).max() <= 2 * math.pi
    assert amp.min() >= 0.5 and amp.max() <= 1.0 and phase.min() >= 0 and phase.max() < 2 * math.pi
    assert np.abs(prob.q.numpy()).max() <= amp.sum(axis=0).max() + 1e-12
    for recipe, n_sets, n_range, e_range in ((inputs.batched_sets_recipe(), 64, (4, 12), (64, 16384)),
                                             (inputs.served_recipe(e_max=2048), 256, (4, 10), (64, 2048))):
        assert len(recipe) == n_sets
        Ns = np.array([r["N"] for r in recipe])
        Es = np.array([r["E"] for r in recipe])
        assert Ns.min() == n_range[0] and Ns.max() == n_range[1]
        assert Es.min() >= e_range[0] and Es.max() <= e_range[1]
        # log-uniform sizes: the median sits near the geometric mean of the range
        gm = math.sqrt(e_range[0] * e_range[1])
        assert gm / 2.5 < np.median(Es) < gm * 2.5
        for r in recipe:
            G = r["grid"][0]
            assert G ** 3 >= r["E"] > (G - 1) ** 3 and r["h"] == 1.0 / G
    t, ids = inputs.served_arrivals(20000, rate=2000.0, n_sims=256, seed=1006)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * 2000.0 - 1.0) < 0.03
    assert ids.min() == 0 and ids.max() == 255
