"""Failure detection on the GPU without a fault: the bounded device-side wait
(the poll loop of the tensor-core kernel's MMA completion wait) runs out on a
barrier nothing arrives at, the kernel sets a status bit and returns, the host
reads STP_ERR_TIMEOUT, and the context stays usable for the next STP."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300 import _binding
from paper_2003_12787_gb300.inputs import elastic_problem

pytestmark = pytest.mark.gpu


def test_wait_runs_out_reports_timeout_and_the_context_stays_usable():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()
    lib = _binding.load()
    prob = elastic_problem(4, E=16, device="cuda")
    with stp.Predictor(3, prob.h, prob.dt) as P:
        stream = torch.cuda.current_stream()
        stp.stp_selftest_bounded_wait(P.handle, 1000, stream)
        flags = ctypes.c_uint()
        status = lib.stp_device_status(P.handle, ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.byref(flags))
        assert status == _binding.STP_ERR_TIMEOUT and flags.value == 2
        # the read cleared the word; the next STP on the same context is right
        avg, faces = P.predict(prob.q, prob.params)
        assert P.status() == 0
        a_ref, f_ref = oracle.stp(prob.q.cpu().numpy(), prob.params.cpu().numpy(), prob.h, prob.dt)
        a = avg.cpu().numpy()
        assert np.abs(a - a_ref).max() <= 1e-12 * np.abs(a_ref).max()
        with pytest.raises(stp.STPError):
            stp.stp_selftest_bounded_wait(P.handle, 0, stream)  # polls out of range
