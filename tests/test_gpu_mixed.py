"""GPU parity of the reduced-precision STP variants against the FP64 oracle:
the split-precision tensor-core variants and the FP32 CUDA-core variant.

Stated error bars (normwise per output array, max|gpu - oracle| / max|oracle|)
on the seeded plane-wave inputs. At order 9 (N=10, the mixed-precision
workload): BF16x3, FP16x2 and FP16x3 <= 1e-9; BF16x2 (16 significant bits
per operand) <= 1e-7. Over N = 2..12 the same bars hold except FP16x2, which
is stated at 2e-9 (measured up to 1.1e-9 at N = 8). The first CK term is
computed in FP64, the later terms on the tensor cores with FP32 accumulation;
the FP32 accumulation sets the ~1e-10 floor. The FP32 variant (same FP64
first term, later terms from FP32 FMA chains) is held to 1e-9 at every N.
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

TOL = {"bf16x2": 1e-7, "bf16x3": 1e-9, "fp16x2": 1e-9, "fp16x3": 1e-9, "fp32": 1e-9}  # order 9
TOL_ANY_N = dict(TOL, fp16x2=2e-9)


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


@pytest.mark.parametrize("precision", list(TOL))
@pytest.mark.parametrize("N", [2, 4, 6, 8, 10, 12])
def test_mixed_parity_small(precision, N):
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5,
                           seed_material=300 + N, seed_waves=400 + N)
    avg, faces = run(prob, precision)
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt)
    errs = errors(avg, faces, a_ref, f_ref)
    assert max(errs) <= TOL_ANY_N[precision], errs
    # the time-dependent part is really computed (not just q passed through)
    assert rel(avg - prob.q.numpy(), a_ref - prob.q.numpy()) < 1e-3


@pytest.mark.parametrize("precision", list(TOL))
def test_mixed_order9_16384_elements_sampled(precision):
    """Order 9 (N=10), 32x32x16 elements of side 1/32, one launch, sampled."""
    prob = elastic_problem(10, grid=(32, 32, 16), h=1.0 / 32, device="cuda")
    rng = np.random.default_rng(9)
    idx = np.unique(np.concatenate([[0, prob.E - 1], rng.choice(prob.E, 40, replace=False)]))
    avg, faces = run(prob, precision, idx)
    it = torch.as_tensor(idx, device="cuda")
    a_ref, f_ref = oracle.stp(prob.q[it].cpu().numpy(), prob.params[it].cpu().numpy(),
                              prob.h, prob.dt)
    errs = errors(avg, faces, a_ref, f_ref)
    assert max(errs) <= TOL[precision], errs


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_mixed_constant_state_exact(precision):
    N, E = 8, 3
    prob = elastic_problem(N, E=E)
    prob.q = prob.q[:, :1, :1, :1, :].expand(E, N, N, N, 9).contiguous()
    avg, faces = run(prob, precision)
    assert rel(avg, prob.q.numpy()) <= 1e-13


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
