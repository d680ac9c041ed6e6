"""Host-side argument checks of the torch wrappers (CPU): shapes, dtypes and
contiguity of q, params and metric are refused before the C ABI is called.
The checks are exercised on a stand-in object, since creating a Predictor
needs a GPU."""
from __future__ import annotations

import types

import pytest
import torch

import paper_2003_12787_gb300 as stp


def _stand_in(N):
    return types.SimpleNamespace(N=N)


def test_inputs_are_checked_before_the_abi():
    N, E = 4, 3
    me = _stand_in(N)
    q = torch.zeros((E, N, N, N, 9), dtype=torch.float64)
    p = torch.zeros((E, N, N, N, 3), dtype=torch.float64)
    stp.Predictor._check_inputs(me, q, p)  # well formed
    bad = [
        (q.float(), p, TypeError),
        (q, p.float(), TypeError),
        (q[..., :8], p, ValueError),                       # 8 quantities
        (q, p[..., :2], ValueError),                       # 2 material parameters
        (q[:2], p, ValueError),                            # element counts differ
        (torch.zeros((E, N, N, N + 1, 9), dtype=torch.float64), p, ValueError),
        (q.transpose(1, 2), p, ValueError),                # not contiguous
        (q, p.transpose(1, 3), ValueError),
        (q.reshape(E, -1), p, ValueError),                 # flattened
    ]
    for qq, pp, err in bad:
        with pytest.raises(err):
            stp.Predictor._check_inputs(me, qq, pp)


def test_metric_is_checked_before_the_abi():
    N, E = 3, 2
    me = _stand_in(N)
    q = torch.zeros((E, N, N, N, 9), dtype=torch.float64)
    m = torch.zeros((E, N, N, N, 3, 3), dtype=torch.float64)
    stp.Predictor._check_metric(me, q, m)
    stp.Predictor._check_metric(me, q, m.reshape(E, N, N, N, 9))  # [..][9] is accepted
    for bad in (m.float(), m[:1], m.transpose(-1, -2), torch.zeros((E, N, N, N, 3, 2),
                                                                    dtype=torch.float64)):
        with pytest.raises(ValueError):
            stp.Predictor._check_metric(me, q, bad)
