"""The C ABI from a plain C program (tests/c/abi_host_predict.c): compiled
with gcc against include/stp.h and linked to the library alone (no CUDA
headers, no Python in the process that computes), it runs the STP through
stp_predict_host; the outputs are checked against the oracle."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300.inputs import elastic_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("N,E", [(4, 37), (8, 5)])
def test_plain_c_program_through_the_abi(tmp_path, N, E):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = stp.build.build()
    exe = tmp_path / "abi_host_predict"
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_host_predict.c"), "-o", str(exe),
                    "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    prob = elastic_problem(N, E=E, seed_material=4000 + N, seed_waves=4100 + N)
    q, params = prob.q.numpy(), prob.params.numpy()
    q.tofile(tmp_path / "q.bin")
    params.tofile(tmp_path / "params.bin")
    r = subprocess.run([str(exe), str(N - 1), repr(prob.h), repr(prob.dt), str(E),
                        str(tmp_path / "q.bin"), str(tmp_path / "params.bin"),
                        str(tmp_path / "avg.bin"), str(tmp_path / "faces.bin")],
                       capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
    avg = np.fromfile(tmp_path / "avg.bin").reshape(E, N, N, N, 9)
    faces = np.fromfile(tmp_path / "faces.bin").reshape(E, 6, N, N, 9)
    a_ref, f_ref = oracle.stp(q, params, prob.h, prob.dt)
    assert rel(avg, a_ref) <= 1e-12 and rel(faces, f_ref) <= 1e-12
