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
from paper_2003_12787_gb300.inputs import curvilinear_problem, elastic_problem, served_arrivals

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


def test_served_workload_at_bench_size_sampled_against_oracle():
    """The served workload as the benchmark runs it: 256 simulations (orders
    3-9, 64-2048 elements each, seed 1005) behind a 2 GiB device pool with 3
    slots, driven by Poisson arrivals at 2000 req/s (seed 1006), so that
    admissions and evictions run all the time. Afterwards sampled elements of
    sampled simulations are stepped by the oracle as often as the server
    stepped them (q_{n+1} := avg_n): the predictor is element-local, so each
    element's trajectory depends on that element alone."""
    import oracle
    from paper_2003_12787_gb300.inputs import served_arrivals, served_recipe
    recipe = served_recipe(e_max=2048)
    budget = 2 << 30
    srv = stp.Server(budget, slots=3)
    rng = np.random.default_rng(11)
    # two sampled simulations per order, three elements each (first, last, one drawn)
    picked = set()
    for N in range(4, 11):
        cand = [i for i, r in enumerate(recipe) if r["N"] == N]
        picked.update(rng.choice(cand, min(2, len(cand)), replace=False).tolist())
    samples, preds = {}, []
    for i, r in enumerate(recipe):
        prob = elastic_problem(r["N"], grid=r["grid"], E=r["E"], h=r["h"],
                               seed_material=r["seed_material"], seed_waves=r["seed_waves"],
                               device="cuda")
        P = stp.Predictor(r["N"] - 1, prob.h, prob.dt)
        assert srv.add_sim(P, prob.q, prob.params) == i
        preds.append(P)
        if i in picked:
            idx = np.unique([0, r["E"] - 1, int(rng.integers(r["E"]))])
            it = torch.as_tensor(idx, device="cuda")
            samples[i] = (idx, prob.q[it].cpu().numpy(), prob.params[it].cpu().numpy(),
                          prob.h, prob.dt)
        del prob
    n_req = 3000
    t, ids = served_arrivals(n_req, rate=2000.0, n_sims=len(recipe), seed=1006)
    lat, wall = srv.run_trace(t, ids)
    assert np.all(np.isfinite(lat)) and np.all(lat > 0) and wall > 0
    st = srv.stats()
    assert st["completed"] == n_req
    assert st["evictions"] > 0 and st["pool_bytes_peak"] <= budget
    counts = np.bincount(ids, minlength=len(recipe))
    checked = 0
    for i, (idx, q_s, p_s, h, dt) in samples.items():
        q, faces, n = srv.read(i)
        assert n == counts[i]
        if n == 0:
            continue
        for _ in range(n):
            avg_ref, faces_ref = oracle.stp(q_s, p_s, h, dt)
            q_s = avg_ref
        tol = 1e-12
        got_q = q[idx].numpy()
        got_f = faces[idx].numpy()
        scale = np.abs(avg_ref).max()
        assert np.abs(got_q - avg_ref).max() <= tol * scale, (i, n)
        for f in range(6):
            s = np.abs(faces_ref[:, f]).max()
            assert np.abs(got_f[:, f] - faces_ref[:, f]).max() <= tol * s, (i, n, f)
        checked += 1
    assert checked >= 12
    srv.close()
    for P in preds:
        P.close()


def _repeated_predict(P, prob, steps):
    """Reference: `steps` single-set predictor calls with q_{n+1} := avg_n."""
    q = prob.q.cuda() if not prob.q.is_cuda else prob.q.clone()
    pa = prob.params.cuda()
    for _ in range(steps):
        q, faces = P.predict(q, pa)
    torch.cuda.synchronize()
    return q.cpu(), faces.cpu()


def test_device_added_simulations_start_resident_and_survive_evictions():
    """Simulations added from device buffers are copied straight into the
    pool while it has room (no pinned copies); the later ones get pinned copies
    at once, the early ones on their first eviction. Every result equals the
    repeated single-set call bit for bit."""
    sims = []
    for i, (N, E) in enumerate(SPECS):
        prob = elastic_problem(N, E=E, seed_material=1900 + i, seed_waves=1950 + i, device="cuda")
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    budget = max(footprint(N, E) for N, E in SPECS) * 2 + (1 << 20)
    srv = stp.Server(budget, slots=3)
    ids = [srv.add_sim(P, prob.q, prob.params) for P, prob in sims]
    steps = 3
    order = np.tile(np.arange(len(sims)), steps)
    t = np.linspace(0.0, 0.01, len(order))
    srv.run_trace(t, np.asarray(ids, dtype=np.int32)[order])
    assert srv.stats()["evictions"] > 0
    for sid, (P, prob) in zip(ids, sims):
        q, faces, n = srv.read(sid)
        q_ref, f_ref = _repeated_predict(P, prob, steps)
        assert n == steps and torch.equal(q, q_ref) and torch.equal(faces, f_ref), sid
    srv.close()
    for P, _ in sims:
        P.close()


def test_ready_order_does_not_change_results():
    """FIFO and resident-first orders run the same requests in other batches:
    each simulation's result is the same bit for bit."""
    sims = problems()
    budget = max(footprint(N, E) for N, E in SPECS) * 2 + (1 << 20)
    t, ids = served_arrivals(60, rate=3000.0, n_sims=len(sims), seed=77)
    out = []
    for policy in (0, 1):
        srv = stp.Server(budget, slots=3)
        srv.set_policy(policy, 0.002)
        sid = [srv.add_sim(P, prob.q, prob.params) for P, prob in sims]
        srv.run_trace(t - t[0], np.asarray(sid, dtype=np.int32)[ids])
        out.append([srv.read(i) for i in sid])
        srv.close()
    for (qa, fa, na), (qb, fb, nb) in zip(*out):
        assert na == nb and torch.equal(qa, qb) and torch.equal(fa, fb)
    for P, _ in sims:
        P.close()


def test_policy_arguments_are_checked():
    srv = stp.Server(1 << 24, slots=1)
    for bad in ((2, 0.1), (1, -1.0), (1, float("inf"))):
        with pytest.raises(stp.STPError):
            srv.set_policy(*bad)
    srv.set_policy(0)
    srv.close()


def test_full_size_simulations_same_alone_and_in_the_mix():
    """Simulations of the full-size served recipe's extremes (order 9 on
    32768 elements, 6.8 GB of pool; order 6 on 20000; order 3 on 64; order 8
    on 5000), added from device buffers: the results of a mixed trace equal
    each simulation run alone bit for bit, and sampled elements of the largest
    one match the oracle stepped as often."""
    import oracle
    specs = [(10, 32768), (7, 20000), (4, 64), (9, 5000)]
    probs = [elastic_problem(N, E=E, seed_material=2100 + i, seed_waves=2150 + i, device="cuda")
             for i, (N, E) in enumerate(specs)]
    preds = [stp.Predictor(p.N - 1, p.h, p.dt) for p in probs]
    steps = [2, 3, 4, 2]
    budget = 40 * 10 ** 9
    alone = []
    for P, prob, n in zip(preds, probs, steps):
        srv = stp.Server(budget, slots=2)
        sid = srv.add_sim(P, prob.q, prob.params)
        for _ in range(n):
            srv.submit(sid)
        srv.drain()
        alone.append(srv.read(sid))
        srv.close()
    srv = stp.Server(budget, slots=3)
    ids = [srv.add_sim(P, prob.q, prob.params) for P, prob in zip(preds, probs)]
    order = np.concatenate([np.full(n, i) for i, n in enumerate(steps)])
    np.random.default_rng(5).shuffle(order)
    t = np.linspace(0.0, 0.02, len(order))
    srv.run_trace(t, np.asarray(ids, dtype=np.int32)[order])
    for sid, (qa, fa, na) in zip(ids, alone):
        q, faces, n = srv.read(sid)
        assert n == na and torch.equal(q, qa) and torch.equal(faces, fa), sid
    q_big = srv.read(ids[0])[0]
    srv.close()
    prob = probs[0]
    idx = [0, 12345, prob.E - 1]
    qs = prob.q[idx].cpu().numpy()
    for _ in range(steps[0]):
        qs, _f = oracle.stp(qs, prob.params[idx].cpu().numpy(), prob.h, prob.dt)
    got = q_big[idx].numpy()
    assert float(np.abs(got - qs).max() / np.abs(qs).max()) <= 1e-12
    for P in preds:
        P.close()


def _served_sources(N, E, rng):
    return [{"element": e, "position": tuple(rng.uniform(0, 1, 3)),
             "amplitude": rng.uniform(-1, 1, 9) * 50.0, "derivatives": rng.uniform(-2, 2, N)}
            for e in (0, E - 1)]


def test_point_sources_in_served_simulations_match_the_oracle():
    """A served simulation with point sources: every step adds the sources'
    response, so after `steps` requests its state equals the oracle's STP with
    sources applied step by step (q_{n+1} = avg_n), within the FP64 bar; the
    same holds alone and in a mix with simulations without sources under a
    budget that evicts, bit for bit."""
    import oracle
    rng = np.random.default_rng(4100)
    steps = 3
    sims = problems()
    srcs = [_served_sources(prob.N, prob.E, rng) if i % 2 == 0 else None
            for i, (P, prob) in enumerate(sims)]
    # alone
    alone = []
    for (P, prob), src in zip(sims, srcs):
        srv = stp.Server(1 << 30, slots=2)
        sid = srv.add_sim(P, prob.q, prob.params, sources=src)
        for _ in range(steps):
            srv.submit(sid)
        srv.drain()
        alone.append(srv.read(sid))
        srv.close()
    # the oracle, step by step
    for (P, prob), src, (q_s, f_s, n) in zip(sims, srcs, alone):
        assert n == steps
        q = prob.q.cpu().numpy()
        for _ in range(steps):
            q, faces = oracle.stp(q, prob.params.cpu().numpy(), prob.h, prob.dt, sources=src)
        s_q, s_f = np.abs(q).max(), np.abs(faces).max()
        assert np.abs(q_s.numpy() - q).max() <= 1e-12 * s_q, prob.N
        assert np.abs(f_s.numpy() - faces).max() <= 1e-12 * s_f, prob.N
    # in the mix, with evictions
    budget = max(footprint(N, E) for N, E in SPECS) * 2 + (1 << 20)
    srv = stp.Server(budget, slots=3)
    ids = [srv.add_sim(P, prob.q, prob.params, sources=src) for (P, prob), src in zip(sims, srcs)]
    order = np.tile(np.arange(len(sims)), steps)
    t = np.linspace(0.0, 0.02, len(order))
    srv.run_trace(t, np.asarray(ids, dtype=np.int32)[order])
    for i, sid in enumerate(ids):
        q_m, f_m, n = srv.read(sid)
        assert n == steps
        assert torch.equal(q_m, alone[i][0]) and torch.equal(f_m, alone[i][1]), i
    assert srv.stats()["evictions"] > 0
    srv.close()


def test_served_source_arguments_are_checked():
    P, prob = problems()[0]
    srv = stp.Server(1 << 28, slots=1)
    N = prob.N
    good = {"element": 0, "position": (0.5, 0.5, 0.5), "amplitude": [1.0] * 9, "derivatives": [1.0] * N}
    for bad in (dict(good, element=prob.E), dict(good, position=(0.5, 1.5, 0.5)),
                dict(good, amplitude=[np.nan] * 9), dict(good, derivatives=[np.inf] * N)):
        with pytest.raises(RuntimeError):
            srv.add_sim(P, prob.q, prob.params, sources=[bad])
    sid = srv.add_sim(P, prob.q, prob.params, sources=[good])
    assert sid == 0  # the failed registrations left no simulation behind
    srv.close()


def test_curvilinear_simulations_with_sources_match_the_oracle():
    """The paper's LOH1 setting in the served loop: curvilinear FP64
    simulations, half of them with point sources, share the persistent
    launch with Cartesian ones. Alone, each equals the oracle's curvilinear
    STP with its sources applied step by step (q_{n+1} = avg_n) within the
    FP64 bar; in the mix, under a budget that evicts, each equals its run
    alone bit for bit."""
    import oracle
    rng = np.random.default_rng(4400)
    steps = 3
    specs = [(4, 40, True), (7, 10, True), (10, 4, True), (6, 20, False), (12, 2, True)]
    sims, srcs = [], []
    for i, (N, E, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=4500 + i, seed_waves=4600 + i)
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
        srcs.append(_served_sources(N, E, rng) if i % 2 == 0 else None)
    alone = []
    for (P, prob), src in zip(sims, srcs):
        srv = stp.Server(1 << 30, slots=2)
        sid = srv.add_sim(P, prob.q, prob.params, metric=prob.metric, sources=src)
        for _ in range(steps):
            srv.submit(sid)
        srv.drain()
        alone.append(srv.read(sid))
        srv.close()
    for (P, prob), src, (q_s, f_s, n) in zip(sims, srcs, alone):
        assert n == steps
        q = prob.q.cpu().numpy()
        for _ in range(steps):
            if prob.metric is not None:
                q, faces = oracle.stp_curvilinear(q, prob.params.numpy(), prob.metric.numpy(), prob.dt,
                                                  sources=src)
            else:
                q, faces = oracle.stp(q, prob.params.numpy(), prob.h, prob.dt, sources=src)
        assert np.abs(q_s.numpy() - q).max() <= 1e-12 * np.abs(q).max(), prob.N
        assert np.abs(f_s.numpy() - faces).max() <= 1e-12 * np.abs(faces).max(), prob.N
    foot = max(8 * E * ((30 if c else 21) * N ** 3 + 54 * N ** 2) + 5 * 256 for N, E, c in specs)
    srv = stp.Server(2 * foot + (1 << 20), slots=3)
    ids = [srv.add_sim(P, prob.q, prob.params, metric=prob.metric, sources=src)
           for (P, prob), src in zip(sims, srcs)]
    order = np.tile(np.arange(len(sims)), steps)
    srv.run_trace(np.linspace(0.0, 0.02, len(order)), np.asarray(ids, dtype=np.int32)[order])
    assert srv.stats()["evictions"] > 0
    for i, sid in enumerate(ids):
        q_m, f_m, n = srv.read(sid)
        assert n == steps
        assert torch.equal(q_m, alone[i][0]) and torch.equal(f_m, alone[i][1]), specs[i]
    srv.close()
    for P, _ in sims:
        P.close()


def _stepped(P, prob, steps):
    q = prob.q.cuda()
    m = prob.metric.cuda() if prob.metric is not None else None
    for _ in range(steps):
        q, faces = P.predict(q, prob.params.cuda(), metric=m)
    torch.cuda.synchronize()
    return q.cpu(), faces.cpu()


def test_large_batches_run_per_shape_and_match_single_set_calls():
    """A batch with more than about 50 ms of FP64 work (eight order-9 sets of
    2000 elements, a curvilinear order-7 set, an order-11 set) runs as
    per-shape persistent launches; served twice, every simulation equals
    repeated single-set calls bit for bit."""
    specs = [(10, 2000, False)] * 8 + [(8, 3000, True), (12, 40, False)]
    sims = []
    for i, (N, E, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=8100 + i, seed_waves=8200 + i, device="cuda")
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    srv = stp.Server(6 << 30, slots=1)
    ids = [srv.add_sim(P, prob.q, prob.params, metric=prob.metric) for P, prob in sims]
    steps = 2
    for _ in range(steps):
        for sid in ids:
            srv.submit(sid)
        srv.drain()
    assert srv.stats()["launches"] == steps  # all ten in one batch per step
    for (P, prob), sid in zip(sims, ids):
        q_s, f_s, n = srv.read(sid)
        assert n == steps
        q_r, f_r = _stepped(P, prob, steps)
        assert torch.equal(q_s, q_r) and torch.equal(f_s, f_r), prob.N
    srv.close()
    for P, _ in sims:
        P.close()


def test_order_11_simulations_round_alike_in_small_batches():
    """In a small batch the order-11 (N = 12) simulation takes the per-shape
    launch while the others share one allocation-free launch; each still
    equals repeated single-set calls bit for bit."""
    specs = [(12, 6), (5, 40), (9, 12)]
    sims = []
    for i, (N, E) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=8300 + i, seed_waves=8400 + i)
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    srv = stp.Server(1 << 30, slots=2)
    ids = [srv.add_sim(P, prob.q, prob.params) for P, prob in sims]
    steps = 3
    for _ in range(steps):
        for sid in ids:
            srv.submit(sid)
        srv.drain()
    for (P, prob), sid in zip(sims, ids):
        q_s, f_s, n = srv.read(sid)
        assert n == steps
        q_r, f_r = _stepped(P, prob, steps)
        assert torch.equal(q_s, q_r) and torch.equal(f_s, f_r), prob.N
    srv.close()
    for P, _ in sims:
        P.close()
