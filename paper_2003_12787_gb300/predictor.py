"""Handle wrapper for torch tensors (allocation of outputs; no arithmetic)."""
from __future__ import annotations

import torch

from . import _binding as B


class Predictor:
    """Owns one stp_handle for (order, dx, dt) on the current CUDA device.
    nodes: "gl" (Gauss-Legendre, default) or "gll" (Gauss-Lobatto)."""

    def __init__(self, order: int, dx: float, dt: float, m: int = 9, precision="fp64",
                 nodes="gl"):
        self.order = order
        self.N = order + 1
        self.dx = dx
        self.dt = dt
        self.nodes = nodes
        self.handle = B.stp_create(order, m, dx, dt, nodes)
        self.precision = precision
        if precision != "fp64":
            B.stp_set_precision(self.handle, precision)

    def status(self, stream=None) -> int:
        """Synchronise and read the device status word (raises STPError on a timeout)."""
        return B.stp_device_status(self.handle, stream)

    def close(self):
        if self.handle is not None:
            B.stp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def empty_outputs(self, E: int, device="cuda", pin_memory: bool = False):
        N = self.N
        if str(device) == "cpu":
            avg = torch.empty((E, N, N, N, 9), dtype=torch.float64, pin_memory=pin_memory)
            faces = torch.empty((E, 6, N, N, 9), dtype=torch.float64, pin_memory=pin_memory)
        else:
            avg = torch.empty((E, N, N, N, 9), dtype=torch.float64, device=device)
            faces = torch.empty((E, 6, N, N, 9), dtype=torch.float64, device=device)
        return avg, faces

    def face_params(self, params: torch.Tensor, stream=None) -> torch.Tensor:
        """Face projection of the material, [E][6][N][N][3] (stp_face_params)."""
        N = self.N
        if params.dtype != torch.float64 or params.dim() != 5 or tuple(params.shape[1:]) != (N, N, N, 3):
            raise ValueError(f"params must be float64 [E][{N}][{N}][{N}][3]")
        if not params.is_contiguous():
            raise ValueError("params must be contiguous")
        out = torch.empty((params.shape[0], 6, N, N, 3), dtype=torch.float64, device=params.device)
        if stream is None and params.is_cuda:
            stream = torch.cuda.current_stream(params.device)
        B.stp_face_params(self.handle, params.shape[0], params, out, stream)
        return out

    def _check_grid(self, grid, q: torch.Tensor):
        gx, gy, gz = (int(g) for g in grid)
        if gx * gy * gz != q.shape[0]:
            raise ValueError(f"grid {tuple(grid)} holds {gx * gy * gz} elements, q has {q.shape[0]}")

    def correct(self, grid, q, params, face_params, avg, faces, out=None, stream=None):
        """Corrector step on the periodic grid (stp_correct); returns q(t + dt).
        out may be q (in place)."""
        self._check_inputs(q, params)
        self._check_grid(grid, q)
        q_out = torch.empty_like(q) if out is None else out
        if stream is None and q.is_cuda:
            stream = torch.cuda.current_stream(q.device)
        B.stp_correct(self.handle, grid, q, params, face_params, avg, faces, q_out, stream)
        return q_out

    def ader_steps(self, grid, q, params, face_params, steps: int, work=None, stream=None):
        """`steps` full ADER-DG steps (predictor + corrector) in place on q
        (stp_ader_step); work = (avg, faces) buffers or None."""
        self._check_inputs(q, params)
        self._check_grid(grid, q)
        avg, faces = work if work is not None else self.empty_outputs(q.shape[0], device=q.device)
        if stream is None and q.is_cuda:
            stream = torch.cuda.current_stream(q.device)
        B.stp_ader_step(self.handle, grid, steps, q, params, face_params, avg, faces, stream)
        return q

    def _check_inputs(self, q: torch.Tensor, params: torch.Tensor):
        N = self.N
        if q.dtype != torch.float64 or params.dtype != torch.float64:
            raise TypeError("q and params must be float64")
        if q.dim() != 5 or tuple(q.shape[1:]) != (N, N, N, 9):
            raise ValueError(f"q must be [E][{N}][{N}][{N}][9], got {tuple(q.shape)}")
        if tuple(params.shape) != (q.shape[0], N, N, N, 3):
            raise ValueError(f"params must be [E][{N}][{N}][{N}][3], got {tuple(params.shape)}")
        if not (q.is_contiguous() and params.is_contiguous()):
            raise ValueError("q and params must be contiguous")

    def predict(self, q: torch.Tensor, params: torch.Tensor, out=None, stream=None, sources=None,
                metric=None):
        """Enqueue on `stream` (default: torch's current stream) for device tensors.
        sources: optional point sources (see stp_predict_sources).
        metric: optional [E][N][N][N][3][3] (or [..][9]) float64 inverse
        Jacobians dxi_d/dx_j of curvilinear elements (stp_predict_curvilinear)."""
        self._check_inputs(q, params)
        E = q.shape[0]
        avg, faces = out if out is not None else self.empty_outputs(E, device=q.device)
        if stream is None and q.is_cuda:
            stream = torch.cuda.current_stream(q.device)
        if metric is not None:
            self._check_metric(q, metric)
            if sources:
                B.stp_predict_sources_curvilinear(self.handle, E, q, params, metric, avg, faces,
                                                  sources, stream)
            else:
                B.stp_predict_curvilinear(self.handle, E, q, params, metric, avg, faces, stream)
        elif sources:
            B.stp_predict_sources(self.handle, E, q, params, avg, faces, sources, stream)
        else:
            B.stp_predict(self.handle, E, q, params, avg, faces, stream)
        return avg, faces

    def _check_metric(self, q: torch.Tensor, metric: torch.Tensor):
        N, E = self.N, q.shape[0]
        if metric.dtype != torch.float64 or not metric.is_contiguous() or \
                metric.numel() != E * N ** 3 * 9 or metric.shape[:4] != q.shape[:4] or \
                metric.device != q.device:
            raise ValueError(f"metric must be a contiguous float64 [E][{N}][{N}][{N}][3][3] "
                             "on the device of q")

    def predict_host(self, q: torch.Tensor, params: torch.Tensor, out=None, stream=None,
                     metric=None):
        """Host tensors in and out (pinned gives full copy bandwidth); synchronous.
        metric: optional host inverse Jacobians of curvilinear elements."""
        self._check_inputs(q, params)
        E = q.shape[0]
        avg, faces = out if out is not None else self.empty_outputs(E, device="cpu")
        if metric is not None:
            self._check_metric(q, metric)
            B.stp_predict_curvilinear_host(self.handle, E, q, params, metric, avg, faces, stream)
        else:
            B.stp_predict_host(self.handle, E, q, params, avg, faces, stream)
        return avg, faces


class Batch:
    """A captured batched launch over several (Predictor, q, params) sets.

    Outputs are allocated here (device tensors) and baked into the plan; each
    launch() replays the plan's CUDA graph on the given stream.
    """

    def __init__(self, items, shapes=None, metrics=None, sources=None):
        """items: (Predictor, q, params) per set; metrics: optional list with
        each set's metric tensor (curvilinear) or None (Cartesian); sources:
        optional list with each set's point sources (list of source dicts as
        for predict, or None)."""
        self.items = []
        sets = []
        for i, (P, q, params) in enumerate(items):
            P._check_inputs(q, params)
            if metrics is not None and metrics[i] is not None:
                P._check_metric(q, metrics[i])
            E = q.shape[0]
            avg, faces = P.empty_outputs(E, device=q.device)
            self.items.append((P, q, params, avg, faces))
            sets.append((P.handle, E, q, params, avg, faces))
        self.metrics = metrics  # keeps the tensors alive with the plan
        if sources is not None:
            if shapes is not None:
                raise ValueError("shapes and sources cannot be combined")
            self.handle = B.stp_batch_create_sources(sets, sources, [it[0].N for it in self.items],
                                                     metrics)
        else:
            self.handle = B.stp_batch_create(sets, shapes, metrics)

    def launch(self, stream=None):
        if stream is None:
            stream = torch.cuda.current_stream()
        B.stp_batch_launch(self.handle, stream)

    def outputs(self, i):
        return self.items[i][3], self.items[i][4]

    def info(self):
        return B.stp_batch_info(self.handle)

    def close(self):
        if self.handle is not None:
            B.stp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The served predictor (continuous batching over resident simulations)."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 3):
        self.handle = B.stp_server_create(hbm_budget_bytes, slots)
        self.budget, self.slots = hbm_budget_bytes, slots
        self.sims = []  # (Predictor, E)
        self._steps0 = []  # steps taken before a restore

    def add_sim(self, predictor: "Predictor", q0: torch.Tensor, params: torch.Tensor,
                metric=None, sources=None) -> int:
        """metric: optional inverse Jacobians (curvilinear simulation);
        sources: optional point sources (as for ``predict_sources``), whose
        response is added after every step."""
        predictor._check_inputs(q0, params)
        if metric is not None:
            predictor._check_metric(q0, metric)
        sid = B.stp_server_add_sim(self.handle, predictor.handle, q0.shape[0], q0, params, metric,
                                   sources)
        self.sims.append((predictor, q0.shape[0]))
        self._steps0.append(0)
        return sid

    def snapshot(self) -> list:
        """Drain, then copy every simulation's state to host memory: a list of
        dicts (q, faces, steps) that ``restore`` turns into a new server in
        the same state."""
        return [dict(zip(("q", "faces", "steps"), self.read(i))) for i in range(len(self.sims))]

    @classmethod
    def restore(cls, snapshot: list, sims: list, hbm_budget_bytes: int, slots: int = 3) -> "Server":
        """A server holding the simulations of ``snapshot``; ``sims`` gives,
        in the same order, (Predictor, params, metric or None[, sources]) of
        each (the inputs that do not change between steps)."""
        if len(snapshot) != len(sims):
            raise ValueError("one (Predictor, params, metric) per snapshot entry")
        srv = cls(hbm_budget_bytes, slots)
        for rec, spec in zip(snapshot, sims):
            P, params, metric = spec[:3]
            sources = spec[3] if len(spec) > 3 else None
            dev = params.device
            srv.add_sim(P, rec["q"].to(dev).contiguous(), params,
                        metric=None if metric is None else metric.to(dev), sources=sources)
            srv._steps0[-1] = int(rec["steps"])
        return srv

    def set_policy(self, policy: int, age_bound_s: float = 0.05):
        """Ready order of the scheduler: 0 FIFO, 1 resident first (default)."""
        B.stp_server_set_policy(self.handle, policy, age_bound_s)

    def submit(self, sim_id: int):
        B.stp_server_submit(self.handle, sim_id)

    def drain(self):
        B.stp_server_drain(self.handle)

    def run_trace(self, t_arrival, sim_ids):
        import numpy as np
        t = np.ascontiguousarray(t_arrival, dtype=np.float64)
        ids = np.ascontiguousarray(sim_ids, dtype=np.int32)
        lat = np.zeros(len(t), dtype=np.float64)
        wall = B.stp_server_run_trace(self.handle, t, ids, lat)
        return lat, wall

    def read(self, sim_id: int):
        P, E = self.sims[sim_id]
        N = P.N
        q = torch.empty((E, N, N, N, 9), dtype=torch.float64)
        faces = torch.empty((E, 6, N, N, 9), dtype=torch.float64)
        steps = B.stp_server_read(self.handle, sim_id, q, faces)
        return q, faces, steps + self._steps0[sim_id]

    def stats(self) -> dict:
        return B.stp_server_stats(self.handle)

    def close(self):
        if self.handle is not None:
            B.stp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
