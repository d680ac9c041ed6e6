"""GPU tests of the served predictor: continuous batching over resident
simulations with HBM-budget admission (and eviction) must give every
simulation exactly the result it gets alone, and the same as repeated
single-set stp_predict calls with q_{n+1} := avg_n."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import elastic_problem, served_arrivals

pytestmark = pytest.mark.gpu

SPECS = [(4, 50), (7, 12), (10, 6), (5, 30), (8, 9), (6, 20)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()


def problems():
    out = []
    for i, (N, E) in enumerate(SPECS):
        prob = elastic_problem(N, E=E, seed_material=900 + i, seed_waves=950 + i)
        out.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    return out


def footprint(N, E):
    return 8 * E * (21 * N ** 3 + 54 * N ** 2) + 4 * 256


def test_same_alone_and_in_the_mix_with_evictions():
    sims = problems()
    steps = 3
    # alone: one simulation per server, big budget
    alone = []
    for P, prob in sims:
        srv = stp.Server(1 << 30, slots=2)
        sid = srv.add_sim(P, prob.q, prob.params)
        for _ in range(steps):
            srv.submit(sid)
        srv.drain()
        alone.append(srv.read(sid))
        srv.close()
    # mixed: all simulations, a budget that holds only about two of them
    budget = max(footprint(N, E) for N, E in SPECS) * 2 + (1 << 20)
    srv = stp.Server(budget, slots=3)
    ids = [srv.add_sim(P, prob.q, prob.params) for P, prob in sims]
    order = np.tile(np.arange(len(sims)), steps)
    t = np.linspace(0.0, 0.02, len(order))
    lat, wall = srv.run_trace(t, np.asarray(ids, dtype=np.int32)[order])
    assert np.all(lat > 0) and wall > 0
    st = srv.stats()
    assert st["completed"] == len(order)
    assert st["evictions"] > 0 and st["pool_bytes_peak"] <= budget
    for i, (P, prob) in enumerate(sims):
        q_mix, f_mix, n_mix = srv.read(ids[i])
        q_al, f_al, n_al = alone[i]
        assert n_mix == n_al == steps
        assert torch.equal(q_mix, q_al) and torch.equal(f_mix, f_al)
        # the same as stepping with the single-set entry point
        q = prob.q.cuda()
        params = prob.params.cuda()
        for _ in range(steps):
            avg, faces = P.predict(q, params)
            q = avg
        torch.cuda.synchronize()
        assert torch.equal(q.cpu(), q_mix) and torch.equal(faces.cpu(), f_mix)
    srv.close()


def test_poisson_trace_completes_with_latencies():
    sims = problems()
    srv = stp.Server(1 << 30, slots=3)
    for P, prob in sims:
        srv.add_sim(P, prob.q, prob.params)
    t, ids = served_arrivals(200, rate=2000.0, n_sims=len(sims), seed=7)
    lat, wall = srv.run_trace(t, ids)
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    st = srv.stats()
    assert st["completed"] == 200 and st["launches"] <= 200
    srv.close()


def test_budget_rejects_a_simulation_that_cannot_fit():
    (P, prob), = problems()[:1]
    srv = stp.Server(1 << 16, slots=1)
    with pytest.raises(stp.STPError):
        srv.add_sim(P, prob.q, prob.params)
    srv.close()


def test_snapshot_and_restore_resume_bit_for_bit():
    """Checkpoint/resume of the served loop: a snapshot after two steps per
    simulation, restored into a new server that runs two more, ends in the
    state of a server that ran four steps without interruption."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_12787_gb300.inputs import curvilinear_problem
    specs = [(5, 20, False), (7, 9, True), (4, 30, False)]
    probs, preds = [], []
    for i, (N, E, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=4200 + i, seed_waves=4300 + i)
        probs.append(prob)
        preds.append(stp.Predictor(N - 1, prob.h, prob.dt))
    budget = 64 << 20

    def run(srv, steps):
        order = np.tile(np.arange(len(specs)), steps)
        srv.run_trace(np.linspace(0.0, 0.005, len(order)), order.astype(np.int32))

    full = stp.Server(budget, slots=2)
    for P, prob in zip(preds, probs):
        full.add_sim(P, prob.q, prob.params, metric=prob.metric)
    run(full, 4)
    first = stp.Server(budget, slots=2)
    for P, prob in zip(preds, probs):
        first.add_sim(P, prob.q, prob.params, metric=prob.metric)
    run(first, 2)
    snap = first.snapshot()
    first.close()
    resumed = stp.Server.restore(snap, [(P, prob.params, prob.metric) for P, prob in zip(preds, probs)],
                                 budget, slots=2)
    run(resumed, 2)
    for i in range(len(specs)):
        q_a, f_a, n_a = full.read(i)
        q_b, f_b, n_b = resumed.read(i)
        assert n_a == n_b == 4
        assert torch.equal(q_a, q_b) and torch.equal(f_a, f_b), specs[i]
    full.close()
    resumed.close()
    for P in preds:
        P.close()
