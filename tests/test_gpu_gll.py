"""GPU parity on Gauss-Lobatto nodes (Sec. II-A allows Gauss-Legendre or
Gauss-Lobatto interpolation points) against the FP64 oracle on the same
family. The kernels are the Gauss-Legendre ones (the node family only changes
the tables), so this checks the tables, their upload and the face vectors,
which are unit vectors here: each face projection is the layer of the average
on that face.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import elastic_problem

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ff": 1e-12, "fp32": 2e-9}


def rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()


def run(prob, precision="fp64", nodes="gll"):
    with stp.Predictor(prob.N - 1, prob.h, prob.dt, precision=precision, nodes=nodes) as P:
        assert stp.stp_get_nodes(P.handle) == stp.NODE_FAMILIES[nodes]
        avg, faces = P.predict(prob.q.cuda(), prob.params.cuda())
        torch.cuda.synchronize()
    return avg.cpu().numpy(), faces.cpu().numpy()


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_gll_fp64_parity_every_order(N):
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5, seed_material=800 + N,
                           seed_waves=900 + N, nodes="gll")
    avg, faces = run(prob)
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt, nodes="gll")
    assert rel(avg, a_ref) <= TOL["fp64"]
    for f in range(6):
        assert rel(faces[:, f], f_ref[:, f]) <= TOL["fp64"]
    # the faces are the boundary layers of the average (unit face vectors)
    assert np.array_equal(faces[:, 0], avg[:, :, :, 0, :])       # x-, [z][y]
    assert np.array_equal(faces[:, 5], avg[:, N - 1, :, :, :])   # z+, [y][x]


@pytest.mark.parametrize("precision,N", [("ff", 4), ("ff", 8), ("ff", 12), ("fp32", 6),
                                         ("fp32", 10)])
def test_gll_other_precisions(precision, N):
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=4, seed_material=820 + N,
                           seed_waves=920 + N, nodes="gll")
    avg, faces = run(prob, precision)
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt, nodes="gll")
    errs = [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]
    assert max(errs) <= TOL[precision], errs


def test_gll_and_gl_sets_in_one_batch():
    """A batch mixing node families (and orders): each set equals its own
    stp_predict bit for bit."""
    specs = [(4, 20, "gll"), (8, 7, "gl"), (8, 5, "gll"), (12, 2, "gll"), (10, 3, "gl")]
    items, probs = [], []
    for i, (N, E, nodes) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=840 + i, seed_waves=940 + i, device="cuda",
                               nodes=nodes)
        P = stp.Predictor(N - 1, prob.h, prob.dt, nodes=nodes)
        items.append((P, prob.q, prob.params))
        probs.append(prob)
    b = stp.Batch(items)
    b.launch()
    torch.cuda.synchronize()
    for i, (P, q, params) in enumerate(items):
        a_b, f_b = b.outputs(i)
        a_s, f_s = P.predict(q, params)
        torch.cuda.synchronize()
        assert torch.equal(a_b, a_s) and torch.equal(f_b, f_s), specs[i]
    b.close()
    for P, _, _ in items:
        P.close()


def test_gll_simulations_in_the_served_loop():
    """Gauss-Lobatto and Gauss-Legendre simulations served together under a
    budget that forces evictions: each equals repeated stp_predict with
    q_{n+1} := avg_n, bit for bit."""
    specs = [(5, 24, "gll"), (8, 9, "gl"), (7, 12, "gll"), (4, 40, "gll")]
    sims = []
    for i, (N, E, nodes) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=860 + i, seed_waves=960 + i, nodes=nodes)
        sims.append((stp.Predictor(N - 1, prob.h, prob.dt, nodes=nodes), prob))
    foot = max(8 * E * (21 * N ** 3 + 54 * N ** 2) for N, E, _ in specs)
    srv = stp.Server(2 * foot + (1 << 20), slots=2)
    ids = [srv.add_sim(P, prob.q, prob.params) for P, prob in sims]
    steps = 3
    order = np.tile(np.arange(len(sims)), steps)
    srv.run_trace(np.linspace(0.0, 0.01, len(order)), np.asarray(ids, dtype=np.int32)[order])
    assert srv.stats()["evictions"] > 0
    for i, (P, prob) in enumerate(sims):
        q_mix, f_mix, n = srv.read(ids[i])
        assert n == steps
        q = prob.q.cuda()
        for _ in range(steps):
            avg, faces = P.predict(q, prob.params.cuda())
            q = avg
        torch.cuda.synchronize()
        assert torch.equal(q.cpu(), q_mix) and torch.equal(faces.cpu(), f_mix), specs[i]
    srv.close()
    for P, _ in sims:
        P.close()
