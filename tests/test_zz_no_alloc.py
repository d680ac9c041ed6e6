"""The allocation-free batched launch (stp_batch_run_static), through the C ABI.

It exists for callers that cannot call cudaMalloc where they run the
predictor: its scratch lives in a fixed array in the library's device image.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test. It must pass both alone in a
fresh process and after the other tests (the array keeps whatever the last
call left in it).
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

TOL = 1e-12  # the FP64 bar of the other parity tests


def rel(a, b):
    s = float(b.abs().max())
    return float((a - b).abs().max()) / (s if s > 0 else 1.0)


def test_static_batch_matches_stp_predict_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()
    # orders 11 and 12 exercise the per-CTA parking areas of the scratch array
    specs = [(4, 37), (12, 3), (11, 2), (8, 9), (1, 5), (10, 4), (6, 17)]
    sets, refs, outs = [], [], []
    for i, (N, E) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=700 + i, seed_waves=800 + i, device="cuda")
        P = stp.Predictor(N - 1, prob.h, prob.dt)
        ref = P.predict(prob.q, prob.params)  # the existing entry point
        avg, faces = P.empty_outputs(E)
        sets.append((P, prob))
        refs.append(ref)
        outs.append((avg, faces))
    torch.cuda.synchronize()
    for call in range(2):
        for avg, faces in outs:
            avg.fill_(float("nan"))
            faces.fill_(float("nan"))
        stp.stp_batch_run_static([(P.handle, prob.E, prob.q, prob.params, a, f)
                                  for (P, prob), (a, f) in zip(sets, outs)])
        torch.cuda.synchronize()
        for (avg, faces), (ra, rf), spec in zip(outs, refs, specs):
            assert rel(avg, ra) <= TOL, (call, spec)
            assert rel(faces, rf) <= TOL, (call, spec)
    # two sets straight against the oracle as well (order 3 whole, and order
    # 11, the order that parks its new Taylor terms in the static array)
    for k in (0, 1):
        (P, prob), (avg, faces) = sets[k], outs[k]
        a_ref, f_ref = oracle.stp(prob.q.cpu().numpy(), prob.params.cpu().numpy(), prob.h, prob.dt)
        assert rel(avg.cpu(), torch.from_numpy(a_ref)) <= TOL, specs[k]
        assert rel(faces.cpu(), torch.from_numpy(f_ref)) <= TOL, specs[k]
    for P, _ in sets:
        P.close()


def test_static_batch_allocates_no_device_memory():
    """After the first call (which loads the module holding the array), a
    call changes the device's free memory by nothing: the entry point takes
    no memory from the device beyond what the library image already holds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    specs = [(12, 2), (8, 3), (4, 20)]
    sets, outs = [], []
    for i, (N, E) in enumerate(specs):
        prob = elastic_problem(N, E=E, seed_material=720 + i, seed_waves=820 + i, device="cuda")
        P = stp.Predictor(N - 1, prob.h, prob.dt)
        sets.append((P, prob))
        outs.append(P.empty_outputs(E))
    args = [(P.handle, prob.E, prob.q, prob.params, a, f) for (P, prob), (a, f) in zip(sets, outs)]
    stp.stp_batch_run_static(args)  # first call: module load, address look-up
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        stp.stp_batch_run_static(args)
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before, (free_before, free_after)
    for P, _ in sets:
        P.close()


def test_static_batch_with_curvilinear_sets():
    """stp_batch_run_static_curvilinear: curvilinear sets of every order in
    the same persistent launch as Cartesian ones (one element per work unit);
    every curvilinear set equals its single-set call bit for bit (the same
    element body and rounding order), the Cartesian ones as in the tests
    above."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    specs = [(N, 3 if N >= 10 else 11, True) for N in range(1, 13)]
    specs += [(8, 9, False), (4, 30, False), (12, 2, False)]
    sets, refs, outs, metrics = [], [], [], []
    for i, (N, E, curv) in enumerate(specs):
        make = curvilinear_problem if curv else elastic_problem
        prob = make(N, E=E, seed_material=900 + i, seed_waves=950 + i, device="cuda")
        P = stp.Predictor(N - 1, prob.h, prob.dt)
        refs.append(P.predict(prob.q, prob.params, metric=prob.metric))
        outs.append(P.empty_outputs(E))
        sets.append((P, prob))
        metrics.append(prob.metric)
    torch.cuda.synchronize()
    stp.stp_batch_run_static([(P.handle, prob.E, prob.q, prob.params, a, f)
                              for (P, prob), (a, f) in zip(sets, outs)], metrics=metrics)
    torch.cuda.synchronize()
    for (avg, faces), (ra, rf), (N, E, curv) in zip(outs, refs, specs):
        if curv or N != 12:
            assert torch.equal(avg, ra) and torch.equal(faces, rf), (N, E, curv)
        else:
            assert rel(avg, ra) <= TOL and rel(faces, rf) <= TOL
    for P, _ in sets:
        P.close()
