"""stp_predict inside a captured CUDA graph: replays give the eager results."""
from __future__ import annotations

import pytest
import torch

import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import elastic_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,precision", [(8, "fp64"), (5, "fp64"), (10, "bf16x3"), (8, "ff"),
                                         (12, "ff"), (10, "fp32")])
def test_predict_captured_in_a_cuda_graph(N, precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()
    prob = elastic_problem(N, E=40, device="cuda", seed_material=60 + N, seed_waves=70 + N)
    with stp.Predictor(N - 1, prob.h, prob.dt, precision=precision) as P:
        ref_a, ref_f = P.predict(prob.q, prob.params)
        torch.cuda.synchronize()
        avg, faces = P.empty_outputs(prob.E)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm-up on the capture stream
            P.predict(prob.q, prob.params, out=(avg, faces), stream=s)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            P.predict(prob.q, prob.params, out=(avg, faces))
        for _ in range(2):
            avg.zero_()
            faces.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(avg, ref_a) and torch.equal(faces, ref_f)
        assert P.status() == 0


def test_orders_and_precisions_mixed_in_one_graph():
    """Several handles of different orders and precisions captured in one
    graph: every replay reproduces each handle's eager results."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()
    cases = [(4, "fp64"), (7, "ff"), (9, "fp32"), (11, "ff")]
    items = []
    for N, precision in cases:
        prob = elastic_problem(N, E=17 + N, device="cuda", seed_material=80 + N, seed_waves=90 + N)
        P = stp.Predictor(N - 1, prob.h, prob.dt, precision=precision)
        ref = P.predict(prob.q, prob.params)
        items.append((P, prob, ref, P.empty_outputs(prob.E)))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for P, prob, _, out in items:
            P.predict(prob.q, prob.params, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for P, prob, _, out in items:
            P.predict(prob.q, prob.params, out=out)
    for _ in range(2):
        for _, _, _, (a, f) in items:
            a.zero_()
            f.zero_()
        g.replay()
        torch.cuda.synchronize()
        for _, _, (ra, rf), (a, f) in items:
            assert torch.equal(a, ra) and torch.equal(f, rf)
    for P, _, _, _ in items:
        P.close()
