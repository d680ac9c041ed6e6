"""GPU parity of the reduced-precision STP variants against the FP64 oracle:
the tensor-core variants (BF16/FP16 digits) and the FP32 CUDA-core variant.

Stated error bars, normwise per output array (max|gpu - oracle| / max|oracle|
over avg and each face array), on seeded plane-wave inputs:

* Tensor-core variants, N <= 10 (float-float steps while a Taylor term is
  above 1e-3 of the state, then the term's contraction as exact products of
  fixed-point digits: up to three 10-bit FP16 digits for FP16x3, two for
  FP16x2, three or two 8-bit BF16 digits for BF16x3 / BF16x2), on resolved
  fields (h = 1/32) AND coarse ones (h = 1/4, 1/5, where the later terms stay
  large): FP16x3 <= 1e-9, FP16x2 <= 5e-8, BF16x3 <= 5e-9, BF16x2 <= 5e-7.
* Tensor-core variants, N = 11, 12 (the earlier kernel: first term in FP64,
  every later term with the variant's slices), resolved fields only:
  BF16x3, FP16x3 <= 1e-9, FP16x2 <= 2e-9, BF16x2 <= 1e-7.
* FP32 (first term in float-float, later terms in FP32): <= 1e-9 on resolved
  fields, <= 1e-8 on coarse ones.

The time-dependent part avg - q (what the predictor adds to the state) is held
to its own bars, relative to max|avg - q| of the oracle.
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

TC = ["bf16x2", "bf16x3", "fp16x2", "fp16x3"]
# resolved fields, N <= 10
TOL = {"bf16x2": 5e-7, "bf16x3": 5e-9, "fp16x2": 5e-8, "fp16x3": 1e-9, "fp32": 1e-9}
# resolved fields, N = 11, 12 (earlier tensor-core kernel)
TOL_N11 = {"bf16x2": 1e-7, "bf16x3": 1e-9, "fp16x2": 2e-9, "fp16x3": 1e-9, "fp32": 1e-9}
# coarse fields, N <= 10
TOL_COARSE = {"bf16x2": 5e-7, "bf16x3": 5e-9, "fp16x2": 5e-8, "fp16x3": 1e-9, "fp32": 1e-8}
# the increment avg - q, relative to its own size
TOL_INCR = {"bf16x2": 1e-5, "bf16x3": 3e-7, "fp16x2": 1e-5, "fp16x3": 3e-7, "fp32": 3e-6}


def rel(a, b):
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    _binding.load()


def run(prob, precision, idx=None):
    q = prob.q if prob.q.is_cuda else prob.q.cuda()
    params = prob.params if prob.params.is_cuda else prob.params.cuda()
    with stp.Predictor(prob.N - 1, prob.h, prob.dt, precision=precision) as P:
        avg, faces = P.predict(q, params)
        assert P.status() == 0
    if idx is not None:
        it = torch.as_tensor(idx, device=avg.device)
        return avg[it].cpu().numpy(), faces[it].cpu().numpy()
    return avg.cpu().numpy(), faces.cpu().numpy()


def errors(avg, faces, a_ref, f_ref):
    return [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]


def check(prob, precision, tol, idx=None):
    avg, faces = run(prob, precision, idx)
    q = prob.q.cpu().numpy() if idx is None else prob.q[torch.as_tensor(idx)].cpu().numpy()
    pa = prob.params.cpu().numpy() if idx is None else prob.params[torch.as_tensor(idx)].cpu().numpy()
    a_ref, f_ref = oracle.stp(q, pa, prob.h, prob.dt)
    errs = errors(avg, faces, a_ref, f_ref)
    assert max(errs) <= tol, errs
    incr = rel(avg - q, a_ref - q)
    assert incr <= TOL_INCR[precision], incr
    return max(errs), incr


@pytest.mark.parametrize("precision", list(TOL))
@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_mixed_parity_resolved(precision, N):
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5,
                           seed_material=300 + N, seed_waves=400 + N)
    check(prob, precision, (TOL if N <= 10 else TOL_N11)[precision])


@pytest.mark.parametrize("precision", list(TOL_COARSE))
@pytest.mark.parametrize("N,h", [(3, 0.25), (5, 0.2), (7, 0.25), (9, 0.2), (10, 0.25), (10, 0.2)])
def test_mixed_parity_coarse(precision, N, h):
    """Coarse fields (the large sets of the batched workload have h = 1/4 ..
    1/9): the later Taylor terms stay large, so more of them need float-float."""
    prob = elastic_problem(N, grid=(4, 4, 4), h=h, E=6, seed_material=500 + N,
                           seed_waves=600 + N)
    check(prob, precision, TOL_COARSE[precision])


@pytest.mark.parametrize("precision", list(TOL))
def test_mixed_order9_16384_elements_sampled(precision):
    """Order 9 (N=10), 32x32x16 elements of side 1/32, one launch, sampled."""
    prob = elastic_problem(10, grid=(32, 32, 16), h=1.0 / 32, device="cuda")
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([[0, prob.E - 1], rng.choice(prob.E, 40, replace=False)]))
    check(prob, precision, TOL[precision], idx)


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x2", "fp32"])
def test_mixed_constant_state_exact(precision):
    N, E = 8, 3
    prob = elastic_problem(N, E=E)
    prob.q = prob.q[:, :1, :1, :1, :].expand(E, N, N, N, 9).contiguous()
    avg, faces = run(prob, precision)
    assert rel(avg, prob.q.numpy()) <= 1e-13


@pytest.mark.parametrize("precision", TC)
def test_zero_state_stays_zero(precision):
    prob = elastic_problem(6, E=4)
    prob.q = torch.zeros_like(prob.q)
    avg, faces = run(prob, precision)
    assert not np.any(avg) and not np.any(faces)


@pytest.mark.parametrize("precision", ["fp16x3", "fp32"])
def test_mixed_host_path_matches_device_path(precision):
    prob = elastic_problem(10, E=40)
    avg_d, faces_d = run(prob, precision)
    with stp.Predictor(9, prob.h, prob.dt, precision=precision) as P:
        avg_h, faces_h = P.predict_host(prob.q.pin_memory(), prob.params.pin_memory())
    assert np.array_equal(avg_h.numpy(), avg_d) and np.array_equal(faces_h.numpy(), faces_d)


def test_precision_setting_round_trip():
    with stp.Predictor(3, 0.1, 0.001) as P:
        assert stp.stp_get_precision(P.handle) == 0
        stp.stp_set_precision(P.handle, "fp16x2")
        assert stp.stp_get_precision(P.handle) == 3
        stp.stp_set_precision(P.handle, "fp32")
        assert stp.stp_get_precision(P.handle) == 5
        with pytest.raises(stp.STPError):
            stp.stp_set_precision(P.handle, 9)
