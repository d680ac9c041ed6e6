"""GPU parity of the corrector and of full ADER-DG steps (predictor +
corrector) against the CPU oracle, through the C ABI.

The bar is the FP64 one of the predictor: max|gpu - oracle| / max|oracle| <=
1e-12 on the corrected state, and on its increment q_out - q separately (the
increment is what the corrector computes; the state passes through).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import paper_2003_12787_gb300 as stp
from paper_2003_12787_gb300.inputs import ader_order7_case, periodic_problem

pytestmark = pytest.mark.gpu

TOL = 1e-12


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    s = float(np.abs(b).max())
    return float(np.abs(a - b).max()) / (s if s > 0 else 1.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stp.build.build()


def _grid_for(N):
    return (3, 2, 2) if N <= 6 else (2, 2, 1) if N <= 10 else (2, 1, 1)


@pytest.mark.parametrize("N", list(range(1, 13)))
def test_corrector_matches_oracle(N):
    grid = _grid_for(N)
    prob = periodic_problem(N, grid, h=0.125, seed_material=300 + N, seed_waves=400 + N,
                            per_node_material=True)
    q, pa = prob.q.numpy(), prob.params.numpy()
    avg, faces = oracle.stp(q, pa, prob.h, prob.dt)
    ref = oracle.correct(q, pa, avg, faces, grid, prob.h, prob.dt)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        qd, pd = prob.q.cuda(), prob.params.cuda()
        fp = P.face_params(pd)
        out = P.correct(grid, qd, pd, fp, torch.from_numpy(avg).cuda(),
                        torch.from_numpy(faces).cuda())
        torch.cuda.synchronize()
    out = out.cpu().numpy()
    assert rel(out, ref) <= TOL, rel(out, ref)
    assert rel(out - q, ref - q) <= TOL, rel(out - q, ref - q)


@pytest.mark.parametrize("N", [1, 4, 7, 12])
def test_face_params_match_oracle(N):
    prob = periodic_problem(N, (2, 2, 2), h=0.25, seed_material=500 + N, per_node_material=True)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        fp = P.face_params(prob.params.cuda())
        torch.cuda.synchronize()
    assert rel(fp.cpu().numpy(), oracle.face_params(prob.params.numpy())) <= 1e-14


@pytest.mark.parametrize("N,grid,steps", [(2, (4, 3, 2), 4), (4, (3, 3, 2), 3), (6, (2, 2, 3), 3),
                                          (8, (2, 2, 2), 3), (11, (2, 1, 2), 2)])
def test_ader_steps_match_oracle(N, grid, steps):
    """Several full steps on the GPU (stp_ader_step: predictor, then corrector
    in place) against the oracle's predictor + corrector steps."""
    prob = periodic_problem(N, grid, h=0.125, seed_material=600 + N, seed_waves=700 + N)
    q0 = prob.q.numpy()
    ref = oracle.ader_steps(q0, prob.params.numpy(), grid, prob.h, prob.dt, steps)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        qd, pd = prob.q.cuda().clone(), prob.params.cuda()
        P.ader_steps(grid, qd, pd, P.face_params(pd), steps)
        torch.cuda.synchronize()
    out = qd.cpu().numpy()
    assert rel(out, ref) <= TOL, rel(out, ref)
    assert rel(out - q0, ref - q0) <= TOL, rel(out - q0, ref - q0)


def test_gauss_lobatto_corrector():
    N, grid = 5, (3, 2, 2)
    prob = periodic_problem(N, grid, h=0.125, seed_material=801, seed_waves=802, nodes="gll",
                            per_node_material=True)
    q0 = prob.q.numpy()
    ref = oracle.ader_steps(q0, prob.params.numpy(), grid, prob.h, prob.dt, 2, nodes="gll")
    with stp.Predictor(N - 1, prob.h, prob.dt, nodes="gll") as P:
        qd, pd = prob.q.cuda().clone(), prob.params.cuda()
        P.ader_steps(grid, qd, pd, P.face_params(pd), 2)
        torch.cuda.synchronize()
    out = qd.cpu().numpy()
    assert rel(out, ref) <= TOL and rel(out - q0, ref - q0) <= TOL


@pytest.mark.parametrize("N,grid", [(3, (1, 1, 1)), (4, (1, 1, 5)), (3, (5, 1, 1)), (5, (1, 3, 1)),
                                    (2, (7, 3, 5))])
def test_degenerate_and_ragged_grids(N, grid):
    """A single element (all six neighbours itself), one-element-thick
    grids, and odd sizes in every direction."""
    prob = periodic_problem(N, grid, h=0.2, seed_material=900 + N, seed_waves=950 + N,
                            per_node_material=True)
    q0 = prob.q.numpy()
    ref = oracle.ader_steps(q0, prob.params.numpy(), grid, prob.h, prob.dt, 2)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        qd, pd = prob.q.cuda().clone(), prob.params.cuda()
        P.ader_steps(grid, qd, pd, P.face_params(pd), 2)
        torch.cuda.synchronize()
    out = qd.cpu().numpy()
    assert rel(out, ref) <= TOL and rel(out - q0, ref - q0) <= TOL


def test_in_place_equals_out_of_place():
    N, grid = 6, (3, 2, 2)
    prob = periodic_problem(N, grid, h=0.125, seed_material=1101, seed_waves=1102)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        qd, pd = prob.q.cuda(), prob.params.cuda()
        fp = P.face_params(pd)
        avg, faces = P.predict(qd, pd)
        out = P.correct(grid, qd, pd, fp, avg, faces)
        qi = qd.clone()
        P.correct(grid, qi, pd, fp, avg, faces, out=qi)
        torch.cuda.synchronize()
    assert torch.equal(out, qi)


def test_constant_state_is_steady_on_the_gpu():
    N, grid = 7, (2, 2, 2)
    prob = periodic_problem(N, grid, h=0.125, seed_material=1201, per_node_material=True)
    q = torch.empty_like(prob.q)
    q[...] = torch.arange(1.0, 10.0, dtype=torch.float64)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        qd, pd = q.cuda(), prob.params.cuda()
        P.ader_steps(grid, qd, pd, P.face_params(pd), 3)
        torch.cuda.synchronize()
    assert rel(qd.cpu().numpy(), q.numpy()) <= 1e-11


def test_argument_errors():
    N, grid = 3, (2, 2, 2)
    prob = periodic_problem(N, grid, h=0.25)
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        qd, pd = prob.q.cuda(), prob.params.cuda()
        fp = P.face_params(pd)
        avg, faces = P.predict(qd, pd)
        with pytest.raises(stp.STPError):  # q_out overlapping avg
            stp.stp_correct(P.handle, grid, qd, pd, fp, avg, faces, avg)
        with pytest.raises(stp.STPError):  # grid dimension 0
            stp.stp_correct(P.handle, (0, 2, 2), qd, pd, fp, avg, faces, qd)
        with pytest.raises(stp.STPError):  # host buffer
            stp.stp_correct(P.handle, grid, prob.q, pd, fp, avg, faces, qd)
        with pytest.raises(stp.STPError):  # negative step count
            stp.stp_ader_step(P.handle, grid, -1, qd, pd, fp, avg, faces)
        with pytest.raises(ValueError):  # grid and q disagree
            P.correct((3, 2, 2), qd, pd, fp, avg, faces)


def _neighbourhood(arr, grid, e):
    """The 27 elements of the 3x3x3 block centred on e (periodic wrap), in the
    element order of a 3x3x3 grid."""
    gx, gy, gz = grid
    ex, ey, ez = e % gx, (e // gx) % gy, e // (gx * gy)
    idx = [((ez + dz) % gz * gy + (ey + dy) % gy) * gx + (ex + dx) % gx
           for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    return arr[idx]


def test_full_size_step_sampled():
    """The benchmark's ADER-DG workload (order 7, periodic 32^3 grid) in the
    launch configuration the benchmark times: one step on the GPU; sampled
    elements checked against the oracle's predictor + corrector on their
    3x3x3 neighbourhood (the corrector of an element reads only its six face
    neighbours, so the centre of the block is an exact subproblem)."""
    prob = ader_order7_case()
    grid = prob.grid
    with stp.Predictor(prob.N - 1, prob.h, prob.dt) as P:
        qd, pd = prob.q.cuda().clone(), prob.params.cuda()
        P.ader_steps(grid, qd, pd, P.face_params(pd), 1)
        torch.cuda.synchronize()
    out = qd.cpu().numpy()
    q, pa = prob.q.numpy(), prob.params.numpy()
    rng = np.random.default_rng(1301)
    samples = [0, prob.E - 1, 31, 32 * 32 - 1] + list(rng.integers(0, prob.E, 4))
    for e in samples:
        qb, pb = _neighbourhood(q, grid, int(e)), _neighbourhood(pa, grid, int(e))
        ref = oracle.ader_steps(qb, pb, (3, 3, 3), prob.h, prob.dt, 1)[13]
        assert rel(out[e], ref) <= TOL, (e, rel(out[e], ref))
        assert rel(out[e] - q[e], ref - q[e]) <= TOL, e
