"""GPU parity of the STP on curvilinear elements against the oracle.

The paper's benchmark meshes are curvilinear (Sec. VI: 9 geometry parameters
per node beside the 3 material parameters). stp_predict_curvilinear takes the
per-node inverse Jacobian dxi_d/dx_j; the oracle applies the chain rule with
dense 9x9 matrices (oracle_stp_curvilinear). FP64 and float-float bar:
normwise 1e-12 per output array.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import curvilinear_problem, elastic_problem

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()


def run(prob, nodes="gl", metric=None, precision="fp64"):
    with stp.Predictor(prob.N - 1, prob.h, prob.dt, nodes=nodes, precision=precision) as P:
        avg, faces = P.predict(prob.q.cuda(), prob.params.cuda(),
                               metric=(prob.metric if metric is None else metric).cuda())
        torch.cuda.synchronize()
    return avg.cpu().numpy(), faces.cpu().numpy()


def check(prob, avg, faces, nodes="gl", idx=None):
    q = prob.q.numpy() if idx is None else prob.q[idx].numpy()
    p = prob.params.numpy() if idx is None else prob.params[idx].numpy()
    m = prob.metric.numpy() if idx is None else prob.metric[idx].numpy()
    a_ref, f_ref = oracle.stp_curvilinear(q, p, m, prob.dt, nodes=nodes)
    errs = [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]
    assert max(errs) <= TOL, errs
    return errs


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_curvilinear_parity_every_order(N):
    """A ragged element count (not a multiple of anything), heterogeneous
    material, a map whose metric varies from node to node."""
    prob = curvilinear_problem(N, grid=(8, 8, 4), E=5 if N >= 9 else 37, seed_material=1500 + N,
                               seed_waves=1600 + N)
    avg, faces = run(prob)
    check(prob, avg, faces)


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_curvilinear_float_float_every_order(N):
    """Float-float (STP_PRECISION_FF) on curvilinear elements: the FP64 bar."""
    prob = curvilinear_problem(N, grid=(8, 8, 4), E=5 if N >= 9 else 37, seed_material=2100 + N,
                               seed_waves=2200 + N)
    avg, faces = run(prob, precision="ff")
    check(prob, avg, faces)


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_curvilinear_fp32_every_order(N):
    """FP32 with a float-float first step on resolved fields (h = 1/32): the
    1e-9-class bar of the Cartesian FP32 variant (2e-9 in the test)."""
    prob = curvilinear_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5 if N >= 9 else 37,
                               seed_material=2500 + N, seed_waves=2600 + N)
    avg, faces = run(prob, precision="fp32")
    a_ref, f_ref = oracle.stp_curvilinear(prob.q.numpy(), prob.params.numpy(),
                                          prob.metric.numpy(), prob.dt)
    errs = [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]
    assert max(errs) <= 2e-9, errs


@pytest.mark.parametrize("N", [4, 9])
def test_curvilinear_float_float_gauss_lobatto_and_scaled_state(N):
    """Gauss-Lobatto nodes, and a state scaled by 2^600 (the per-element
    power-of-two scaling keeps it inside the float range)."""
    prob = curvilinear_problem(N, grid=(8, 8, 4), E=6, seed_material=2300 + N,
                               seed_waves=2400 + N, nodes="gll")
    prob.q = prob.q * 2.0 ** 600
    avg, faces = run(prob, nodes="gll", precision="ff")
    check(prob, avg, faces, nodes="gll")


@pytest.mark.parametrize("N", [2, 5, 8, 12])
def test_curvilinear_gauss_lobatto(N):
    prob = curvilinear_problem(N, grid=(8, 8, 4), E=6, seed_material=1700 + N,
                               seed_waves=1800 + N, nodes="gll")
    avg, faces = run(prob, nodes="gll")
    check(prob, avg, faces, nodes="gll")


@pytest.mark.parametrize("N", [4, 8, 11])
def test_cube_metric_matches_cartesian_path(N):
    """G = I/h: the curvilinear kernel reproduces stp_predict (different
    kernels and rounding order, so to 1e-13, not bitwise)."""
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=9, seed_material=1900 + N,
                           seed_waves=1950 + N)
    G = torch.zeros((prob.E, N, N, N, 3, 3), dtype=torch.float64)
    G[...] = torch.eye(3, dtype=torch.float64) / prob.h
    prob.metric = G
    a_c, f_c = run(prob)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        a, f = P.predict(prob.q.cuda(), prob.params.cuda())
        torch.cuda.synchronize()
    assert rel(a_c, a.cpu().numpy()) <= 1e-13 and rel(f_c, f.cpu().numpy()) <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "ff"])
def test_full_order7_workload_sampled(precision):
    """The benchmark's curvilinear order-7 workload (32^3 elements), in the
    launch the benchmark times; 48 sampled elements against the oracle."""
    prob = curvilinear_problem(8, grid=(32, 32, 32), device="cuda")
    with stp.Predictor(7, prob.h, prob.dt, precision=precision) as P:
        avg, faces = P.predict(prob.q, prob.params, metric=prob.metric)
        torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    idx = np.sort(np.concatenate([[0, prob.E - 1], rng.choice(prob.E, 46, replace=False)]))
    t = torch.as_tensor(idx, device="cuda")
    sub = type(prob)(N=8, E=len(idx), h=prob.h, dt=prob.dt, q=prob.q[t].cpu(),
                     params=prob.params[t].cpu(), grid=prob.grid, metric=prob.metric[t].cpu())
    check(sub, avg[t].cpu().numpy(), faces[t].cpu().numpy())


def test_element_independence_and_graph_capture():
    N = 7
    prob = curvilinear_problem(N, grid=(8, 8, 8), E=300, seed_material=2001, seed_waves=2002,
                               device="cuda")
    perm = torch.randperm(prob.E, generator=torch.Generator().manual_seed(3)).cuda()
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        a, f = P.predict(prob.q, prob.params, metric=prob.metric)
        ap, fp = P.predict(prob.q[perm].contiguous(), prob.params[perm].contiguous(),
                           metric=prob.metric[perm].contiguous())
        s = torch.cuda.Stream()
        out = P.empty_outputs(prob.E)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            P.predict(prob.q, prob.params, out=out, metric=prob.metric)
        g.replay()
        torch.cuda.synchronize()
    assert torch.equal(ap, a[perm]) and torch.equal(fp, f[perm])
    assert torch.equal(out[0], a) and torch.equal(out[1], f)


@pytest.mark.parametrize("precision", ["fp64", "ff", "fp32"])
def test_host_buffer_path_equals_device_path(precision):
    """stp_predict_curvilinear_host (chunked copies and kernels over three
    streams; 1000 elements at N = 8 make three chunks) gives the device
    path's results bit for bit."""
    N = 8
    prob = curvilinear_problem(N, grid=(16, 16, 4), E=1000, seed_material=2701, seed_waves=2702)
    with stp.Predictor(N - 1, prob.h, prob.dt, precision=precision) as P:
        a_d, f_d = P.predict(prob.q.cuda(), prob.params.cuda(), metric=prob.metric.cuda())
        torch.cuda.synchronize()
        a_h, f_h = P.predict_host(prob.q.pin_memory(), prob.params.pin_memory(),
                                  metric=prob.metric.pin_memory())
        # the Cartesian host path on the same handle reuses the (larger)
        # staging buffers of the curvilinear call
        a_c, _ = P.predict_host(prob.q, prob.params)
        a_cd, _ = P.predict(prob.q.cuda(), prob.params.cuda())
        torch.cuda.synchronize()
    assert torch.equal(a_h, a_d.cpu()) and torch.equal(f_h, f_d.cpu())
    assert torch.equal(a_c, a_cd.cpu())


def test_batch_of_curvilinear_and_cartesian_sets():
    """stp_batch_create_curvilinear: curvilinear sets of several orders and
    precisions beside Cartesian ones in one graph plan; each set's results
    equal its own single-set call bit for bit."""
    specs = [(8, 300, "fp64", True), (5, 700, "ff", True), (10, 40, "fp32", True),
             (4, 900, "fp64", False), (7, 120, "ff", False), (12, 9, "fp64", True)]
    items, metrics, probs = [], [], []
    for i, (N, E, prec, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=2800 + i, seed_waves=2900 + i, device="cuda")
        P = stp.Predictor(N - 1, prob.h, prob.dt, precision=prec)
        items.append((P, prob.q, prob.params))
        metrics.append(prob.metric if curv else None)
        probs.append(prob)
    b = stp.Batch(items, metrics=metrics)
    b.launch()
    b.launch()  # a replay gives the same results
    torch.cuda.synchronize()
    for i, (P, q, params) in enumerate(items):
        a_b, f_b = b.outputs(i)
        a_s, f_s = P.predict(q, params, metric=metrics[i])
        torch.cuda.synchronize()
        assert torch.equal(a_b, a_s) and torch.equal(f_b, f_s), specs[i]
    b.close()
    for P, _, _ in items:
        P.close()


def test_fp64_curvilinear_sets_share_the_persistent_launch():
    """An all-FP64 batch with curvilinear sets of every order beside Cartesian
    ones is one persistent launch (units: one per curvilinear element, plus the
    Cartesian element groups); every set equals its single-set call bit for
    bit, replayed twice, and the curvilinear ones also meet the oracle."""
    specs = [(N, 3 if N >= 10 else 7, True) for N in range(1, 13)]
    specs += [(6, 250, False), (9, 40, False), (12, 6, False)]
    items, metrics, probs = [], [], []
    for i, (N, E, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=4200 + i, seed_waves=4300 + i)
        items.append((stp.Predictor(N - 1, prob.h, prob.dt), prob.q.cuda(), prob.params.cuda()))
        metrics.append(prob.metric.cuda() if curv else None)
        probs.append(prob)
    b = stp.Batch(items, metrics=metrics)
    info = b.info()
    assert info["ctas"] > 0, "an all-FP64 batch is one persistent launch"
    assert info["units"] >= sum(E for _, E, c in specs if c)
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    for i, (P, q, params) in enumerate(items):
        a_b, f_b = b.outputs(i)
        a_s, f_s = P.predict(q, params, metric=metrics[i])
        torch.cuda.synchronize()
        assert torch.equal(a_b, a_s) and torch.equal(f_b, f_s), specs[i]
        if specs[i][2] and specs[i][0] in (1, 4, 7, 12):
            check(probs[i], a_b.cpu().numpy(), f_b.cpu().numpy())
    b.close()
    for P, _, _ in items:
        P.close()


def test_curvilinear_simulations_in_the_served_loop():
    """Curvilinear and Cartesian simulations served together under a budget
    that forces evictions (the metric is re-admitted with the state): each
    equals repeated single-set calls with q_{n+1} := avg_n, bit for bit."""
    specs = [(5, 24, True), (8, 9, False), (7, 12, True), (4, 40, True)]
    sims = []
    for i, (N, E, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=3000 + i, seed_waves=3100 + i)
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    foot = max(8 * E * ((30 if c else 21) * N ** 3 + 54 * N ** 2) for N, E, c in specs)
    srv = stp.Server(2 * foot + (1 << 20), slots=2)
    ids = [srv.add_sim(P, prob.q, prob.params, metric=prob.metric) for P, prob in sims]
    steps = 3
    order = np.tile(np.arange(len(sims)), steps)
    srv.run_trace(np.linspace(0.0, 0.01, len(order)), np.asarray(ids, dtype=np.int32)[order])
    assert srv.stats()["evictions"] > 0
    for i, (P, prob) in enumerate(sims):
        q_mix, f_mix, n = srv.read(ids[i])
        assert n == steps
        q = prob.q.cuda()
        m = prob.metric.cuda() if prob.metric is not None else None
        for _ in range(steps):
            avg, faces = P.predict(q, prob.params.cuda(), metric=m)
            q = avg
        torch.cuda.synchronize()
        assert torch.equal(q.cpu(), q_mix) and torch.equal(faces.cpu(), f_mix), specs[i]
    srv.close()
    for P, _ in sims:
        P.close()


def test_other_precisions_in_the_served_loop():
    """Float-float and FP32 simulations (Cartesian and curvilinear) beside
    FP64 ones in the served loop, with evictions: each equals repeated
    single-set calls in its handle's precision, bit for bit."""
    specs = [(6, 30, "ff", False), (8, 9, "fp64", False), (7, 12, "fp32", True),
             (5, 40, "ff", True), (4, 50, "fp32", False)]
    sims = []
    for i, (N, E, prec, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=3700 + i, seed_waves=3800 + i)
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt, precision=prec), prob))
    foot = max(8 * E * ((30 if c else 21) * N ** 3 + 54 * N ** 2) for N, E, _, c in specs)
    srv = stp.Server(2 * foot + (1 << 20), slots=2)
    ids = [srv.add_sim(P, prob.q, prob.params, metric=prob.metric) for P, prob in sims]
    steps = 3
    order = np.tile(np.arange(len(sims)), steps)
    srv.run_trace(np.linspace(0.0, 0.01, len(order)), np.asarray(ids, dtype=np.int32)[order])
    assert srv.stats()["evictions"] > 0
    for i, (P, prob) in enumerate(sims):
        q_mix, f_mix, n = srv.read(ids[i])
        assert n == steps
        q = prob.q.cuda()
        m = prob.metric.cuda() if prob.metric is not None else None
        for _ in range(steps):
            avg, faces = P.predict(q, prob.params.cuda(), metric=m)
            q = avg
        torch.cuda.synchronize()
        assert torch.equal(q.cpu(), q_mix) and torch.equal(faces.cpu(), f_mix), specs[i]
    srv.close()
    for P, _ in sims:
        P.close()


@pytest.mark.parametrize("precision", ["fp64", "ff", "fp32"])
def test_constant_state_is_steady_on_curvilinear_elements(precision):
    """A state constant in each element has zero derivatives along every
    reference direction, whatever the metric: avg = q and every face = q, up
    to the rounding of D's row sums (which are zero in exact arithmetic)."""
    N = 6
    prob = curvilinear_problem(N, grid=(8, 8, 4), E=20, seed_material=3900, seed_waves=3901)
    rng = np.random.default_rng(3902)
    const = torch.from_numpy(rng.uniform(-1, 1, (prob.E, 1, 1, 1, 9)))
    prob.q = const.expand(prob.E, N, N, N, 9).contiguous()
    avg, faces = run(prob, precision=precision)
    q = prob.q.numpy()
    assert np.abs(avg - q).max() <= 1e-12 * np.abs(q).max()
    for f in range(6):
        assert np.abs(faces[:, f] - q[:, 0]).max() <= 1e-12 * np.abs(q).max()


def test_argument_errors():
    N = 4
    prob = curvilinear_problem(N, E=8, device="cuda")
    E = prob.E
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        avg, faces = P.empty_outputs(E)
        h = P.handle
        m = prob.metric
        with pytest.raises(stp.STPError) as ei:
            _binding.stp_predict_curvilinear(h, E, prob.q, prob.params, None, avg, faces)
        assert ei.value.status == _binding.STP_ERR_INVALID_ARG
        with pytest.raises(stp.STPError) as ei:  # metric overlapping an output
            _binding.stp_predict_curvilinear(h, E, prob.q, prob.params, avg, avg, faces)
        assert ei.value.status == _binding.STP_ERR_INVALID_ARG
        with pytest.raises(stp.STPError) as ei:  # host metric
            _binding.stp_predict_curvilinear(h, E, prob.q, prob.params, m.cpu(), avg, faces)
        assert ei.value.status == _binding.STP_ERR_INVALID_ARG
        _binding.stp_predict_curvilinear(h, 0, prob.q, prob.params, None, avg, faces)  # E = 0
        with pytest.raises(ValueError):
            P.predict(prob.q, prob.params, metric=m[:, :, :, :, :2])
        P.predict(prob.q, prob.params, metric=m)  # valid after the errors
        torch.cuda.synchronize()
    for prec in ("fp16x2", "bf16x3"):
        with stp.Predictor(N - 1, prob.h, prob.dt, precision=prec) as P:
            with pytest.raises(stp.STPError) as ei:
                P.predict(prob.q, prob.params, metric=m)
            assert ei.value.status == _binding.STP_ERR_UNSUPPORTED
