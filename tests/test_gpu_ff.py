"""GPU parity of the float-float STP variant (every step in float-float on the
FP32 pipes) against the FP64 oracle.

Stated bar: normwise relative error (max|gpu - oracle| / max|oracle| per
output array) <= 1e-12 for 2 <= N <= 12, the same bar as the FP64 kernel.
The float-float significand has about 48 bits (2^-48 = 3.6e-15); the
contractions add a few units of that per step.

Invariant checked bit for bit: the kernel scales each element's state by a
power of two before the arithmetic, so multiplying q by 2^k multiplies every
output by exactly 2^k (for k far beyond the FP32 exponent range too).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import elastic_problem, order7_case, order9_case

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


def run(prob, precision, q=None, idx=None):
    q = prob.q if q is None else q
    q = q if q.is_cuda else q.cuda()
    params = prob.params if prob.params.is_cuda else prob.params.cuda()
    with stp.Predictor(prob.N - 1, prob.h, prob.dt, precision=precision) as P:
        avg, faces = P.predict(q, params)
    torch.cuda.synchronize()
    if idx is not None:
        it = torch.as_tensor(idx, device=avg.device)
        return avg[it].cpu().numpy(), faces[it].cpu().numpy()
    return avg.cpu().numpy(), faces.cpu().numpy()


def errors(avg, faces, a_ref, f_ref):
    return [rel(avg, a_ref)] + [rel(faces[:, f], f_ref[:, f]) for f in range(6)]


@pytest.mark.parametrize("N", list(range(2, 13)))
def test_ff_parity_every_order(N):
    prob = elastic_problem(N, grid=(32, 32, 16), h=1.0 / 32, E=5,
                           seed_material=500 + N, seed_waves=600 + N)
    avg, faces = run(prob, "ff")
    a_ref, f_ref = oracle.stp(prob.q.numpy(), prob.params.numpy(), prob.h, prob.dt)
    errs = errors(avg, faces, a_ref, f_ref)
    assert max(errs) <= TOL, errs
    assert rel(avg - prob.q.numpy(), a_ref - prob.q.numpy()) < 1e-9


@pytest.mark.parametrize("case", [order7_case, order9_case], ids=["order7_32768", "order9_16384"])
def test_ff_full_workloads_sampled(case):
    prob = case(device="cuda")
    rng = np.random.default_rng(77)
    idx = np.unique(np.concatenate([[0, prob.E - 1], rng.choice(prob.E, 24, replace=False)]))
    avg, faces = run(prob, "ff", idx=idx)
    it = torch.as_tensor(idx, device="cuda")
    a_ref, f_ref = oracle.stp(prob.q[it].cpu().numpy(), prob.params[it].cpu().numpy(),
                              prob.h, prob.dt)
    errs = errors(avg, faces, a_ref, f_ref)
    assert max(errs) <= TOL, errs


@pytest.mark.parametrize("precision", ["ff", "fp32"])
@pytest.mark.parametrize("k", [-700, -140, 90, 700])
def test_power_of_two_scaling_is_exact(precision, k):
    prob = elastic_problem(7, E=6, seed_material=41, seed_waves=42)
    a0, f0 = run(prob, precision)
    a1, f1 = run(prob, precision, q=prob.q * (2.0 ** k))
    assert np.array_equal(a1, a0 * 2.0 ** k)
    assert np.array_equal(f1, f0 * 2.0 ** k)


@pytest.mark.parametrize("N", [4, 8, 11])
def test_ff_rough_random_data(N):
    """Uniform random state and material per node (no smoothness, Taylor
    terms that do not decay): the float-float variant still meets the FP64
    bar."""
    rng = np.random.default_rng(2024 + N)
    E = 6
    q = torch.from_numpy(rng.uniform(-1, 1, (E, N, N, N, 9)))
    params = np.stack([rng.uniform(2, 3, (E, N, N, N)), rng.uniform(4, 6, (E, N, N, N)),
                       rng.uniform(1, 2.5, (E, N, N, N))], axis=-1)
    h = 0.1
    dt = 0.4 * h / ((2 * N - 1) * params[..., 1].max())
    with stp.Predictor(N - 1, h, dt, precision="ff") as P:
        avg, faces = P.predict(q.cuda(), torch.from_numpy(params).cuda())
        torch.cuda.synchronize()
    a_ref, f_ref = oracle.stp(q.numpy(), params, h, dt)
    errs = errors(avg.cpu().numpy(), faces.cpu().numpy(), a_ref, f_ref)
    assert max(errs) <= TOL, errs


def test_ff_constant_state_exact():
    N, E = 9, 3
    prob = elastic_problem(N, E=E)
    prob.q = prob.q[:, :1, :1, :1, :].expand(E, N, N, N, 9).contiguous()
    avg, faces = run(prob, "ff")
    assert rel(avg, prob.q.numpy()) <= 1e-13


def test_ff_host_path_matches_device_path():
    prob = elastic_problem(8, E=37)
    avg_d, faces_d = run(prob, "ff")
    with stp.Predictor(7, prob.h, prob.dt, precision="ff") as P:
        avg_h, faces_h = P.predict_host(prob.q.pin_memory(), prob.params.pin_memory())
    assert np.array_equal(avg_h.numpy(), avg_d) and np.array_equal(faces_h.numpy(), faces_d)


def test_ff_order_11_slot_body_matches_its_own_host_path_and_scaling():
    """N = 12 runs the slot-reusing body: ragged count, host path, exact scaling."""
    prob = elastic_problem(12, E=3, seed_material=71, seed_waves=72)
    a0, f0 = run(prob, "ff")
    a1, f1 = run(prob, "ff", q=prob.q * 2.0 ** -300)
    assert np.array_equal(a1, a0 * 2.0 ** -300) and np.array_equal(f1, f0 * 2.0 ** -300)
    with stp.Predictor(11, prob.h, prob.dt, precision="ff") as P:
        avg_h, faces_h = P.predict_host(prob.q.pin_memory(), prob.params.pin_memory())
    assert np.array_equal(avg_h.numpy(), a0) and np.array_equal(faces_h.numpy(), f0)


def test_ff_unknown_precision_value_is_rejected():
    with stp.Predictor(5, 0.1, 0.001) as P:
        with pytest.raises(stp.STPError):
            stp.stp_set_precision(P.handle, 7)
        assert stp.stp_get_precision(P.handle) == 0
