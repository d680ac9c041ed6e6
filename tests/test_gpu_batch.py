"""GPU tests of the batched persistent launches (mixed orders and sizes, one
persistent kernel per shape replayed from a CUDA graph, autotuned shapes).

Every unit of the batch runs the same per-node FP64 arithmetic as the
single-set kernel, so batched results must equal single-set results bit for
bit, whatever else is in the batch ("same alone and in the mix"), and match
the oracle within the FP64 bar.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import batched_sets_recipe, elastic_problem

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


def make_sets(specs):
    out = []
    for i, (N, E) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=500 + i, seed_waves=600 + i, device="cuda")
        out.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    return out


SPECS = [(4, 37), (12, 3), (2, 130), (7, 11), (10, 4), (5, 64), (1, 9), (9, 5), (11, 2),
         (6, 17), (8, 9), (3, 70)]


def test_batch_matches_single_set_kernel_bitwise_and_oracle():
    sets = make_sets(SPECS)
    b = stp.Batch([(P, prob.q, prob.params) for P, prob in sets])
    b.launch()
    torch.cuda.synchronize()
    info = b.info()
    assert info["units"] > 0 and info["ctas"] > 0
    for i, (P, prob) in enumerate(sets):
        avg_b, faces_b = b.outputs(i)
        avg_s, faces_s = P.predict(prob.q, prob.params)
        torch.cuda.synchronize()
        assert torch.equal(avg_b, avg_s) and torch.equal(faces_b, faces_s), SPECS[i]
        a_ref, f_ref = oracle.stp(prob.q.cpu().numpy(), prob.params.cpu().numpy(), prob.h, prob.dt)
        assert rel(avg_b.cpu().numpy(), a_ref) <= 1e-12
        for f in range(6):
            assert rel(faces_b[:, f].cpu().numpy(), f_ref[:, f]) <= 1e-12
    b.close()


def test_same_alone_and_in_the_mix_and_graph_replay():
    sets = make_sets(SPECS[:6])
    mix = stp.Batch([(P, prob.q, prob.params) for P, prob in sets])
    mix.launch()
    mix.launch()  # a second replay writes the same values again
    torch.cuda.synchronize()
    for i, (P, prob) in enumerate(sets):
        alone = stp.Batch([(P, prob.q, prob.params)])
        alone.launch()
        torch.cuda.synchronize()
        a1, f1 = mix.outputs(i)
        a2, f2 = alone.outputs(i if False else 0)
        assert torch.equal(a1, a2) and torch.equal(f1, f2)
        alone.close()
    mix.close()


def test_batch_of_other_precisions_is_a_graph_of_per_set_launches():
    """Sets in the float-float, FP32, tensor-core and FP64 precisions in one
    plan: every set's outputs equal its own stp_predict bit for bit, on every
    replay; the float-float sets also meet the FP64 bar against the oracle."""
    specs = [(4, 37), (12, 3), (7, 11), (10, 4), (9, 5), (2, 30), (11, 2), (8, 9)]
    precisions = ["ff", "ff", "fp32", "bf16x3", "fp64", "ff", "fp32", "ff"]
    sets = make_sets(specs)
    for (P, _), prec in zip(sets, precisions):
        stp.stp_set_precision(P.handle, prec)
    b = stp.Batch([(P, prob.q, prob.params) for P, prob in sets])
    info = b.info()
    assert info["units"] == len(sets) and info["ctas"] == 0
    for _ in range(2):
        b.launch()
        torch.cuda.synchronize()
        for i, (P, prob) in enumerate(sets):
            avg_b, faces_b = b.outputs(i)
            avg_s, faces_s = P.predict(prob.q, prob.params)
            torch.cuda.synchronize()
            assert torch.equal(avg_b, avg_s) and torch.equal(faces_b, faces_s), (specs[i], precisions[i])
            if precisions[i] == "ff":
                a_ref, f_ref = oracle.stp(prob.q.cpu().numpy(), prob.params.cpu().numpy(),
                                          prob.h, prob.dt)
                assert rel(avg_b.cpu().numpy(), a_ref) <= 1e-12
    b.close()


def test_autotune_reports_candidates():
    for N in (4, 8, 12):
        with stp.Predictor(N - 1, 0.1, 1e-4) as P:
            t = stp.stp_autotune(P.handle)
            assert t["variant"] in (0, 1)
            assert t["us_per_element"] > 0
            assert t["us_variants"][t["variant"]] == t["us_per_element"]
            assert min(u for u in t["us_variants"] if u > 0) == t["us_per_element"]


def test_batch_rejects_bad_sets():
    (P, prob), = make_sets([(4, 8)])
    avg, faces = P.empty_outputs(8)
    with pytest.raises(stp.STPError):  # output aliases an input
        stp.stp_batch_create([(P.handle, 8, prob.q, prob.params, prob.q, faces)])
    with pytest.raises(stp.STPError):  # outputs of two sets overlap
        stp.stp_batch_create([(P.handle, 8, prob.q, prob.params, avg, faces),
                              (P.handle, 8, prob.q, prob.params, avg, faces)])
    M = stp.Predictor(3, prob.h, prob.dt, precision="bf16x3")
    with pytest.raises(stp.STPError):  # shapes apply to all-FP64 batches only
        stp.stp_batch_create([(M.handle, 8, prob.q, prob.params, avg, faces)], shapes=[0])
    mixed = stp.stp_batch_create([(M.handle, 8, prob.q, prob.params, avg, faces)], shapes=[-1])
    stp.stp_batch_destroy(mixed)
    empty = stp.stp_batch_create([(P.handle, 0, prob.q, prob.params, avg, faces)])
    stp.stp_batch_launch(empty)  # nothing to do
    stp.stp_batch_destroy(empty)


def test_batched_workload_64_sets_sampled():
    """64 sets, orders 3-11, 64-16384 elements each (seed 1003), one launch:
    a sample of elements of every set against the oracle."""
    recipe = batched_sets_recipe()
    probs, preds = [], []
    for r in recipe:
        prob = elastic_problem(r["N"], grid=r["grid"], E=r["E"], h=r["h"],
                               seed_material=r["seed_material"], seed_waves=r["seed_waves"],
                               device="cuda")
        probs.append(prob)
        preds.append(stp.Predictor(r["N"] - 1, prob.h, prob.dt))
    b = stp.Batch([(P, prob.q, prob.params) for P, prob in zip(preds, probs)])
    b.launch()
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    worst = 0.0
    for i, prob in enumerate(probs):
        idx = np.unique(np.concatenate([[0, prob.E - 1], rng.choice(prob.E, 2, replace=False)]))
        it = torch.as_tensor(idx, device="cuda")
        a_ref, f_ref = oracle.stp(prob.q[it].cpu().numpy(), prob.params[it].cpu().numpy(),
                                  prob.h, prob.dt)
        avg, faces = b.outputs(i)
        worst = max(worst, rel(avg[it].cpu().numpy(), a_ref))
        for f in range(6):
            worst = max(worst, rel(faces[it][:, f].cpu().numpy(), f_ref[:, f]))
    assert worst <= 1e-12, worst
    b.close()


def test_more_sets_of_one_shape_than_one_launch_holds():
    """A launch carries at most 128 set descriptors (a kernel-parameter table):
    150 sets of one order are split over two launches of the same shape's
    kernel, beside sets of other orders; every set still equals its
    single-set call bit for bit, over two replays, and the plan's units
    cover every element."""
    specs = [(4, 1 + (i % 5)) for i in range(150)] + [(7, 6), (12, 2), (9, 3)]
    sets = []
    for i, (N, E) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=7000 + i, seed_waves=7500 + i, device="cuda")
        sets.append((stp.Predictor(N - 1, prob.h, prob.dt), prob))
    b = stp.Batch([(P, prob.q, prob.params) for P, prob in sets], shapes=[0] * len(specs))
    info = b.info()
    # shape 0 of N = 4 holds 8 elements per unit: one unit per set there
    assert info["units"] == 150 + 6 + 2 + 3
    b.launch()
    b.launch()
    torch.cuda.synchronize()
    for i, (P, prob) in enumerate(sets):
        a_b, f_b = b.outputs(i)
        a_s, f_s = P.predict(prob.q, prob.params)
        torch.cuda.synchronize()
        assert torch.equal(a_b, a_s) and torch.equal(f_b, f_s), specs[i]
    b.close()
    for P, _ in sets:
        P.close()
