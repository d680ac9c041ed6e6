"""GPU parity of the STP with point sources against the oracle.

A point source (a Dirac delta in one element times an amplitude vector times a
time function given by its derivatives) enters every Cauchy-Kowalewsky order,
q^(k+1) = L q^(k) + s^(k). The library adds the sources' response to the
outputs of the elements that hold them (an FP64 launch after the STP); the
oracle adds s^(k) inside its own recurrence. Elements without sources must be
bitwise those of stp_predict.
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


def rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()


def make_sources(N, E, rng, per_element=((1, 3), (4, 1))):
    out = []
    for e, count in per_element:
        if e >= E:
            continue
        for _ in range(count):
            out.append({"element": e, "position": tuple(rng.uniform(0, 1, 3)),
                        "amplitude": rng.uniform(-1, 1, 9) * 50.0,
                        "derivatives": rng.uniform(-2, 2, N)})
    return out


def run(prob, sources, precision="fp64", nodes="gl"):
    with stp.Predictor(prob.N - 1, prob.h, prob.dt, precision=precision, nodes=nodes) as P:
        q, params = prob.q.cuda(), prob.params.cuda()
        a_s, f_s = P.predict(q, params, sources=sources)
        a_0, f_0 = P.predict(q, params)
        torch.cuda.synchronize()
    return a_s.cpu().numpy(), f_s.cpu().numpy(), a_0.cpu().numpy(), f_0.cpu().numpy()


@pytest.mark.parametrize("N,nodes", [(1, "gl"), (2, "gl"), (4, "gl"), (8, "gl"), (12, "gl"),
                                     (5, "gll"), (9, "gll")])
def test_sources_fp64_parity(N, nodes):
    rng = np.random.default_rng(3000 + N)
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5, seed_material=1100 + N,
                           seed_waves=1200 + N, nodes=nodes)
    src = make_sources(N, prob.E, rng)
    avg, faces, avg0, faces0 = run(prob, src, nodes=nodes)
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt, nodes=nodes,
                              sources=src)
    assert rel(avg, a_ref) <= 1e-12
    for f in range(6):
        assert rel(faces[:, f], f_ref[:, f]) <= 1e-12
    # the sources matter, and only in their elements
    assert rel(avg[1], avg0[1]) > 1e-8
    for e in (0, 2, 3):
        assert np.array_equal(avg[e], avg0[e]) and np.array_equal(faces[e], faces0[e])


@pytest.mark.parametrize("precision,tol", [("ff", 1e-12), ("fp32", 2e-9)])
def test_sources_with_other_precisions(precision, tol):
    N = 7
    rng = np.random.default_rng(77)
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=6, seed_material=1300,
                           seed_waves=1301)
    src = make_sources(N, prob.E, rng)
    avg, faces, _, _ = run(prob, src, precision=precision)
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt, sources=src)
    errs = [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]
    assert max(errs) <= tol, errs


def test_source_on_a_gauss_lobatto_corner_node():
    """A source at a corner of a Gauss-Lobatto element projects onto that
    node only (phi is a unit vector there)."""
    N = 4
    rng = np.random.default_rng(5)
    prob = elastic_problem(N, E=2, seed_material=1400, seed_waves=1401, nodes="gll")
    src = [{"element": 0, "position": (0.0, 1.0, 0.0), "amplitude": rng.uniform(-1, 1, 9),
            "derivatives": rng.uniform(-1, 1, N)}]
    avg, faces, _, _ = run(prob, src, nodes="gll")
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt, nodes="gll",
                              sources=src)
    assert rel(avg, a_ref) <= 1e-12 and rel(faces, f_ref) <= 1e-12


def run_curv(prob, sources, precision="fp64", nodes="gl"):
    with stp.Predictor(prob.N - 1, prob.h, prob.dt, precision=precision, nodes=nodes) as P:
        q, params, m = prob.q.cuda(), prob.params.cuda(), prob.metric.cuda()
        a_s, f_s = P.predict(q, params, sources=sources, metric=m)
        a_0, f_0 = P.predict(q, params, metric=m)
        torch.cuda.synchronize()
    return a_s.cpu().numpy(), f_s.cpu().numpy(), a_0.cpu().numpy(), f_0.cpu().numpy()


@pytest.mark.parametrize("N,nodes", [(1, "gl"), (2, "gl"), (5, "gl"), (8, "gl"), (12, "gl"),
                                     (6, "gll")])
def test_sources_on_curvilinear_elements(N, nodes):
    """A point source in a curvilinear mesh (the node volume of the mass
    matrix is w |det J|, taken from the metric on the device)."""
    rng = np.random.default_rng(3300 + N)
    prob = curvilinear_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5, seed_material=3400 + N,
                               seed_waves=3500 + N, nodes=nodes)
    src = make_sources(N, prob.E, rng)
    avg, faces, avg0, faces0 = run_curv(prob, src, nodes=nodes)
    a_ref, f_ref = oracle.stp_curvilinear(prob.q.numpy(), prob.params.numpy(), prob.metric.numpy(),
                                          prob.dt, nodes=nodes, sources=src)
    assert rel(avg, a_ref) <= 1e-12
    for f in range(6):
        assert rel(faces[:, f], f_ref[:, f]) <= 1e-12
    assert rel(avg[1], avg0[1]) > 1e-8
    for e in (0, 2, 3):
        assert np.array_equal(avg[e], avg0[e]) and np.array_equal(faces[e], faces0[e])


@pytest.mark.parametrize("precision,tol", [("ff", 1e-12), ("fp32", 2e-9)])
def test_sources_on_curvilinear_elements_other_precisions(precision, tol):
    N = 7
    rng = np.random.default_rng(78)
    prob = curvilinear_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=6, seed_material=3600,
                               seed_waves=3601)
    src = make_sources(N, prob.E, rng)
    avg, faces, _, _ = run_curv(prob, src, precision=precision)
    a_ref, f_ref = oracle.stp_curvilinear(prob.q.numpy(), prob.params.numpy(), prob.metric.numpy(),
                                          prob.dt, sources=src)
    errs = [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]
    assert max(errs) <= tol, errs


def test_source_argument_errors():
    N = 3
    prob = elastic_problem(N, E=4, device="cuda")
    good = {"element": 1, "position": (0.5, 0.5, 0.5), "amplitude": [1.0] * 9,
            "derivatives": [1.0] * N}
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        for bad in (dict(good, element=4), dict(good, element=-1),
                    dict(good, position=(0.5, 1.5, 0.5)), dict(good, amplitude=[np.nan] * 9),
                    dict(good, derivatives=[np.inf] * N)):
            with pytest.raises(stp.STPError) as ei:
                P.predict(prob.q, prob.params, sources=[good, bad])
            assert ei.value.status == _binding.STP_ERR_INVALID_ARG
        P.predict(prob.q, prob.params, sources=[good])  # valid after the errors
        torch.cuda.synchronize()


BATCH_SPECS = [(4, 30, True), (8, 7, False), (10, 5, True), (6, 12, False), (12, 2, True), (1, 9, True)]


def _batch_problems(seed0):
    rng = np.random.default_rng(seed0)
    out = []
    for i, (N, E, with_src) in enumerate(BATCH_SPECS):
        prob = elastic_problem(N, E=E, seed_material=seed0 + i, seed_waves=seed0 + 50 + i,
                               device="cuda")
        src = make_sources(N, E, rng, per_element=((0, 2), (E - 1, 1))) if with_src else None
        out.append((prob, src))
    return out


def _oracle_set(prob, src):
    q, pa = prob.q.cpu().numpy(), prob.params.cpu().numpy()
    return oracle.stp(q, pa, prob.h, prob.dt, sources=src) if src else oracle.stp(q, pa, prob.h, prob.dt)


@pytest.mark.parametrize("precisions", [("fp64",) * 6, ("fp64", "ff", "fp64", "fp32", "fp64", "fp64")])
def test_batch_plan_with_and_without_sources(precisions):
    """A batch plan mixing sets with and without point sources: every set
    equals the oracle with its sources (FP64 and float-float sets within
    1e-12; the FP32 set within its coarse-field 1e-8), and the sets without sources are
    unchanged by the others'. All-FP64 sets run in the persistent launch,
    the mixed-precision plan as a graph of per-set launches."""
    sets = _batch_problems(4100)
    preds = [stp.Predictor(p.N - 1, p.h, p.dt, precision=prec)
             for (p, _), prec in zip(sets, precisions)]
    b = stp.Batch([(P, p.q, p.params) for P, (p, _) in zip(preds, sets)],
                  sources=[src for _, src in sets])
    for _ in range(2):  # a second replay gives the same result (no accumulation)
        b.launch()
    torch.cuda.synchronize()
    for i, ((prob, src), prec) in enumerate(zip(sets, precisions)):
        a_ref, f_ref = _oracle_set(prob, src)
        avg, faces = b.outputs(i)
        tol = 1e-8 if prec == "fp32" else 1e-12  # FP32 on these coarse cubes: its 1e-8 bar
        assert rel(avg.cpu().numpy(), a_ref) <= tol, (i, prec)
        assert rel(faces.cpu().numpy(), f_ref) <= tol, (i, prec)
    for P in preds:
        P.close()


def test_static_batch_with_and_without_sources():
    """The allocation-free launch with per-set point sources (their data in
    the static array's top): every set equals the oracle within 1e-12, on two
    calls in a row."""
    sets = _batch_problems(4300)
    preds = [stp.Predictor(p.N - 1, p.h, p.dt) for p, _ in sets]
    outs = [P.empty_outputs(p.E) for P, (p, _) in zip(preds, sets)]
    args = [(P.handle, p.E, p.q, p.params, a, f) for P, (p, _), (a, f) in zip(preds, sets, outs)]
    refs = [_oracle_set(p, src) for p, src in sets]
    for call in range(2):
        for a, f in outs:
            a.fill_(float("nan"))
            f.fill_(float("nan"))
        stp.stp_batch_run_static_sources(args, [src for _, src in sets], [p.N for p, _ in sets])
        torch.cuda.synchronize()
        for i, ((a, f), (a_ref, f_ref)) in enumerate(zip(outs, refs)):
            assert rel(a.cpu().numpy(), a_ref) <= 1e-12, (call, i)
            assert rel(f.cpu().numpy(), f_ref) <= 1e-12, (call, i)
    for P in preds:
        P.close()


def test_batch_source_arguments_are_checked():
    prob = elastic_problem(4, E=3, device="cuda")
    P = stp.Predictor(3, prob.h, prob.dt)
    a, f = P.empty_outputs(3)
    bad = [{"element": 5, "position": (0.5, 0.5, 0.5), "amplitude": [1.0] * 9, "derivatives": [1.0] * 4}]
    with pytest.raises(stp.STPError):
        stp._binding.stp_batch_create_sources([(P.handle, 3, prob.q, prob.params, a, f)], [bad], [4])
    with pytest.raises(stp.STPError):
        stp.stp_batch_run_static_sources([(P.handle, 3, prob.q, prob.params, a, f)], [bad], [4])
    P.close()
