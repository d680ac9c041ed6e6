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
