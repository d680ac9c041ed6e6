#!/usr/bin/env python
"""Benchmark of the GB300 Space-Time Predictor.

One step = one STP pass (CK loop, Taylor time average, six face projections)
over the whole workload: order 7 (N=8), 32^3 = 32768 elastic elements of side
1/32, FP64, inputs resident in HBM. Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the plain FP64 CPU oracle on the host cores on a
bounded sample of the same workload per step (the reference arm).
Under torchrun (N > 1) every rank runs its own seeded partition of the same
size (weak scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "STP elements/s + % FP64 roofline; mixed vs FP64 at fixed error; p50/p99"
UNIT = "elements/s"
PROFILES = os.path.join(ROOT, "profiles")

WORKLOADS = {
    # name: (N, grid, h, description)
    "order7": (8, (32, 32, 32), 1.0 / 32,
               "order-7 (N=8) elastic STP, 32^3=32768 elements of side 1/32, one launch"),
    "order3": (4, (8, 8, 8), 1.0 / 8,
               "order-3 (N=4) elastic STP, 8^3=512 elements of side 1/8, one launch"),
    "order7_small": (8, (16, 16, 16), 1.0 / 32,
                     "order-7 (N=8) elastic STP, 16^3=4096 elements of side 1/32, one launch"),
    "order9_small": (10, (16, 16, 8), 1.0 / 32,
                     "order-9 (N=10) elastic STP, 16x16x8=2048 elements of side 1/32, one launch"),
    "order9": (10, (32, 32, 16), 1.0 / 32,
               "order-9 (N=10) elastic STP, 32x32x16=16384 elements of side 1/32, one launch"),
}


def flops_per_element(N: int) -> int:
    """Algorithmic FP64 flops of one element (elastic sparsity, N CK steps):
    36N^5 (derivative contractions) + 48N^4 (pointwise elastic update)
    + 18N^4 (Taylor accumulation) + 108N^3 (six face projections)."""
    return 36 * N ** 5 + 66 * N ** 4 + 108 * N ** 3


def flops_per_element_dense(N: int) -> int:
    """The same count with all 9 quantities differentiated in every direction
    (54N^5 for the contractions instead of 36N^5): stated beside the
    roofline so that avoided work is not counted as done."""
    return 54 * N ** 5 + 66 * N ** 4 + 108 * N ** 3


def flops_per_element_curvilinear(N: int) -> int:
    """Algorithmic FP64 flops of one curvilinear element: per CK step and node,
    27 reference derivatives (54N flops), the chain rule through the metric
    (27 x 3 products added into 9 physical sums: 108 flops, counting only the
    18 nonzero couplings per direction as the elastic system needs them), the
    pointwise update (48) and the average (18); faces as in the Cartesian
    count: 54N^5 + 174N^4 + 108N^3."""
    return 54 * N ** 5 + 174 * N ** 4 + 108 * N ** 3


def bytes_per_element(N: int) -> int:
    """Algorithmic HBM bytes of one element: q (9N^3) + params (3N^3) in,
    avg (9N^3) + faces (54N^2) out, 8 bytes each."""
    return 8 * (21 * N ** 3 + 54 * N ** 2)


# FP64 ALU peak derived from unit counts and clock: 152 SMs x 2 DFMA/clk/SM
# (the FP64 pipe rate of GB300) x 2 flops x 2.07 GHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def kernel_source_hash() -> str:
    """Hash of the sources of the FP64 kernel the bench times."""
    h = hashlib.sha256()
    for name in ("fp64_kernels.cu", "fp64_eo.cuh", "fp64_group.cuh", "ck_fp64.cuh"):
        with open(os.path.join(ROOT, "paper_2003_12787_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_record(workload: str):
    """The committed ncu record of the FP64 kernel on this workload, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(PROFILES, f"traffic_fp64_stp_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha") != kernel_source_hash():
        return None
    return rec


def traffic_from_profile(workload: str):
    """DRAM bytes per launch from the committed ncu record (stored figure, not
    measured in this run), or None."""
    rec = profile_record(workload)
    return None if rec is None else rec.get("dram_bytes_per_launch")


def fp64_pipe_fraction(workload: str, ms_per_launch: float, sm_mhz):
    """Share of the FP64 pipe's issue capacity the kernel used: thread-level
    FP64 instructions per launch (committed ncu record) over 2 per clock per
    SM x 152 SMs x the SM clock sampled during the timed region x the launch
    time. Independent of how many flops an instruction is counted for."""
    rec = profile_record(workload)
    if rec is None or not rec.get("fp64_thread_inst_per_launch") or not sm_mhz:
        return None
    return rec["fp64_thread_inst_per_launch"] / (2 * 152 * sm_mhz * 1e6 * ms_per_launch / 1e3)


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(", ") for l in self.file.read().splitlines() if l.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                power.append(float(r[3]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_model() -> str:
    """The host CPU's name as the OS reports it (model name, else the part)."""
    import platform
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
        for key in ("model name", "Model name", "CPU part"):
            for line in info.splitlines():
                if line.startswith(key):
                    return f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_baseline(prob_q, prob_params, h, dt, budget_s: float, max_elems: int, metric=None):
    """Time the oracle as it stands on a bounded sample (elements from the
    front of the workload, in chunks, until the time budget is spent);
    curvilinear elements when a metric is given."""
    import oracle
    E = prob_q.shape[0]
    done, spent, chunk = 0, 0.0, 256
    while done < min(E, max_elems) and spent < budget_s:
        n = min(chunk, E - done, max_elems - done)
        q = np.ascontiguousarray(prob_q[done:done + n])
        p = np.ascontiguousarray(prob_params[done:done + n])
        t0 = time.perf_counter()
        if metric is None:
            oracle.stp(q, p, h, dt)
        else:
            oracle.stp_curvilinear(q, p, np.ascontiguousarray(metric[done:done + n]), dt)
        spent += time.perf_counter() - t0
        done += n
        chunk = min(chunk * 2, 4096)
    return done, spent, oracle.num_threads()


PRECISIONS_ALL = ("fp64", "ff", "fp32", "bf16x2", "bf16x3", "fp16x2", "fp16x3")


def mixed_comparison(stp, torch, args, workload="order9", precisions=PRECISIONS_ALL):
    """Reduced-precision variants vs FP64 at their measured error on one
    workload (default: order 9, N=10, 16384 elements): per precision, the
    CUDA-event time of one launch (mean of args.mixed_steps after 3 warm-ups)
    and the max normwise error of avg and the six face arrays against the
    oracle on a sample of elements."""
    import oracle
    from paper_2003_12787_gb300.inputs import elastic_problem
    N, grid, h, desc = WORKLOADS[workload]
    prob = elastic_problem(N, grid=grid, h=h, device="cuda")
    E = prob.E
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 14, replace=False)]))
    it = torch.as_tensor(idx, device="cuda")
    a_ref, f_ref = oracle.stp(prob.q[it].cpu().numpy(), prob.params[it].cpu().numpy(),
                              prob.h, prob.dt)
    out = {"workload": desc, "elements": E, "N": N,
           "error": "max over avg and 6 face arrays of max|gpu-oracle|/max|oracle|, "
                    f"{len(idx)} sampled elements", "variants": {}}
    stream = torch.cuda.current_stream()
    for prec in precisions:
        P = stp.Predictor(N - 1, prob.h, prob.dt, precision=prec)
        avg, faces = P.empty_outputs(E)
        for _ in range(3):
            P.predict(prob.q, prob.params, out=(avg, faces), stream=stream)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(args.mixed_steps):
            P.predict(prob.q, prob.params, out=(avg, faces), stream=stream)
        s1.record(stream)
        torch.cuda.synchronize()
        P.status(stream)
        ms = s0.elapsed_time(s1) / args.mixed_steps
        a = avg[it].cpu().numpy()
        f = faces[it].cpu().numpy()
        err = max([float(np.abs(a - a_ref).max() / np.abs(a_ref).max())] +
                  [float(np.abs(f[:, i] - f_ref[:, i]).max() / np.abs(f_ref[:, i]).max())
                   for i in range(6)])
        out["variants"][prec] = {"ms_per_launch": ms, "elements_per_s": E / (ms / 1e3),
                                 "max_rel_err": err,
                                 "tflops_algorithmic": E * flops_per_element(N) / (ms / 1e3) / 1e12}
        P.close()
    base = out["variants"]["fp64"]["ms_per_launch"]
    for v in out["variants"].values():
        v["speedup_vs_fp64"] = base / v["ms_per_launch"]
    return out


def curvilinear_measurement(stp, torch, args, cartesian_ms: float):
    """The order-7 workload on curvilinear elements (the same 32^3 grid pushed
    through a smooth map; 9 more per-node parameters, the inverse Jacobian),
    in FP64, float-float and FP32: CUDA-event time of one
    stp_predict_curvilinear launch (mean of args.mixed_steps after 3
    warm-ups), the algorithmic rate and the error of 12 sampled elements
    against the oracle."""
    import oracle
    from paper_2003_12787_gb300.inputs import curvilinear_problem
    N, grid, h, _ = WORKLOADS["order7"]
    prob = curvilinear_problem(N, grid=grid, h=h, device="cuda")
    E = prob.E
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(8)
    idx = np.unique(np.concatenate([[0, E - 1], rng.choice(E, 10, replace=False)]))
    it = torch.as_tensor(idx, device="cuda")
    a_ref, f_ref = oracle.stp_curvilinear(prob.q[it].cpu().numpy(), prob.params[it].cpu().numpy(),
                                          prob.metric[it].cpu().numpy(), prob.dt)
    out = {"workload": "order-7 (N=8) elastic STP on curvilinear elements, 32^3=32768 "
                       "elements, smooth map of amplitude 0.2, one launch",
           "elements": E, "flops_per_element": flops_per_element_curvilinear(N),
           "error": f"max over avg and 6 face arrays, {len(idx)} sampled elements vs the oracle",
           "variants": {}}
    for prec in ("fp64", "ff", "fp32"):
        with stp.Predictor(N - 1, prob.h, prob.dt, precision=prec) as P:
            avg, faces = P.empty_outputs(E)
            for _ in range(3):
                P.predict(prob.q, prob.params, out=(avg, faces), stream=stream, metric=prob.metric)
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.mixed_steps):
                P.predict(prob.q, prob.params, out=(avg, faces), stream=stream, metric=prob.metric)
            s1.record(stream)
            torch.cuda.synchronize()
            ms = s0.elapsed_time(s1) / args.mixed_steps
        a = avg[it].cpu().numpy()
        f = faces[it].cpu().numpy()
        err = max([float(np.abs(a - a_ref).max() / np.abs(a_ref).max())] +
                  [float(np.abs(f[:, i] - f_ref[:, i]).max() / np.abs(f_ref[:, i]).max())
                   for i in range(6)])
        tf = E * flops_per_element_curvilinear(N) / (ms / 1e3) / 1e12
        out["variants"][prec] = {
            "ms_per_launch": ms, "elements_per_s": E / (ms / 1e3), "tflops_algorithmic": tf,
            "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS,
            "hbm_gbs": E * 8 * (30 * N ** 3 + 54 * N ** 2) / (ms / 1e3) / 1e9,
            "time_vs_cartesian_fp64": ms / cartesian_ms, "max_rel_err": err}
    for prec in ("ff", "fp32"):
        out["variants"][prec]["speedup_vs_fp64"] = (out["variants"]["fp64"]["ms_per_launch"] /
                                                    out["variants"][prec]["ms_per_launch"])
    # the paper's own setting for its headline figure: N = 11 (order 10) on
    # curvilinear elements; 4096 elements of side 1/32 on the smooth map
    N11 = 11
    p11 = curvilinear_problem(N11, grid=(16, 16, 16), h=1.0 / 32, device="cuda")
    out["order10"] = {"workload": "order-10 (N=11) elastic STP on curvilinear elements, "
                                  "16^3=4096 elements of side 1/32, one launch",
                      "flops_per_element": flops_per_element_curvilinear(N11), "variants": {}}
    for prec in ("fp64", "ff"):
        with stp.Predictor(N11 - 1, p11.h, p11.dt, precision=prec) as P:
            avg, faces = P.empty_outputs(p11.E)
            for _ in range(3):
                P.predict(p11.q, p11.params, out=(avg, faces), stream=stream, metric=p11.metric)
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.mixed_steps):
                P.predict(p11.q, p11.params, out=(avg, faces), stream=stream, metric=p11.metric)
            s1.record(stream)
            torch.cuda.synchronize()
            ms = s0.elapsed_time(s1) / args.mixed_steps
        tf = p11.E * flops_per_element_curvilinear(N11) / (ms / 1e3) / 1e12
        out["order10"]["variants"][prec] = {"ms_per_launch": ms,
                                            "elements_per_s": p11.E / (ms / 1e3),
                                            "tflops_algorithmic": tf,
                                            "frac_of_fp64_peak": tf / FP64_PEAK_TFLOPS}
    return out


def small_case_latency(stp, torch, args):
    """The small order-3 workload (N=4, 8^3 = 512 elements, 31 MFLOP): a
    latency-bound launch. Per launch, the device time (CUDA events around
    it) and the host launch-to-done time (stp_predict call to stream
    synchronisation), 5 warm-ups then args.small_launches timed; p50/p99.
    Then the same launch captured once into a CUDA graph: host replay-to-done
    time of the replays (argument checks and launch set-up paid once)."""
    from paper_2003_12787_gb300.inputs import elastic_problem
    N, grid, h, desc = WORKLOADS["order3"]
    prob = elastic_problem(N, grid=grid, h=h, device="cuda")
    stream = torch.cuda.current_stream()
    dev, host = [], []
    with stp.Predictor(N - 1, prob.h, prob.dt) as P:
        avg, faces = P.empty_outputs(prob.E)
        for i in range(5 + args.small_launches):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            P.predict(prob.q, prob.params, out=(avg, faces), stream=stream)
            e1.record(stream)
            stream.synchronize()
            t1 = time.perf_counter()
            if i >= 5:
                dev.append(e0.elapsed_time(e1) * 1e3)
                host.append((t1 - t0) * 1e6)

        # the same launch captured once into a CUDA graph: replay cost only
        gstream = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=gstream):
            P.predict(prob.q, prob.params, out=(avg, faces))
        graph_host = []
        for i in range(5 + args.small_launches):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.replay()
            torch.cuda.current_stream().synchronize()
            t1 = time.perf_counter()
            if i >= 5:
                graph_host.append((t1 - t0) * 1e6)

    def pct(v, p):
        return float(np.percentile(np.array(v), p))
    return {"workload": desc, "launches": args.small_launches,
            "device_us": {"p50": pct(dev, 50), "p99": pct(dev, 99)},
            "launch_to_done_us": {"p50": pct(host, 50), "p99": pct(host, 99)},
            "graph_replay_to_done_us": {"p50": pct(graph_host, 50), "p99": pct(graph_host, 99)},
            "elements_per_s_p50": prob.E / (pct(dev, 50) * 1e-6)}


def batched_measurement(stp, torch, args):
    """The batched workload (64 sets, orders 3-11, 64-16384 elements each,
    seed 1003) as one persistent launch per shape, replayed from a CUDA graph: time per
    replay (CUDA events, mean of args.batch_steps after one warm-up), element
    throughput, algorithmic FP64 rate, and the autotuner's choice per order."""
    from paper_2003_12787_gb300.inputs import batched_sets_recipe, elastic_problem
    recipe = batched_sets_recipe(e_max=args.batched_emax)
    items, flops, elems = [], 0, 0
    for r in recipe:
        prob = elastic_problem(r["N"], grid=r["grid"], E=r["E"], h=r["h"],
                               seed_material=r["seed_material"], seed_waves=r["seed_waves"],
                               device="cuda")
        items.append((stp.Predictor(r["N"] - 1, prob.h, prob.dt), prob.q, prob.params))
        flops += r["E"] * flops_per_element(r["N"])
        elems += r["E"]
    t0 = time.perf_counter()
    b = stp.Batch(items)
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    b.launch(stream)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("batched_timed")
    s0.record(stream)
    for _ in range(args.batch_steps):
        b.launch(stream)
    s1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = s0.elapsed_time(s1) / args.batch_steps
    tuned = {}
    for P, _, _ in items:
        if P.N not in tuned:
            tuned[P.N] = stp.stp_autotune(P.handle)
    # the same sets in the float-float and FP32 variants: a graph of per-set
    # launches; error of element 0 of every set against the oracle
    import oracle
    refs = [oracle.stp(q[:1].cpu().numpy(), pr[:1].cpu().numpy(), P.dx, P.dt) for P, q, pr in items]
    variants = {}
    for prec in ("ff", "fp32"):
        for P, _, _ in items:
            stp.stp_set_precision(P.handle, prec)
        bv = stp.Batch(items)
        bv.launch(stream)
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        for _ in range(args.batch_steps):
            bv.launch(stream)
        v1.record(stream)
        torch.cuda.synchronize()
        vms = v0.elapsed_time(v1) / args.batch_steps
        err = 0.0
        for i, (a_ref, f_ref) in enumerate(refs):
            a, f = bv.outputs(i)
            a = a[:1].cpu().numpy()
            f = f[:1].cpu().numpy()
            err = max(err, float(np.abs(a - a_ref).max() / np.abs(a_ref).max()),
                      max(float(np.abs(f[:, j] - f_ref[:, j]).max() / np.abs(f_ref[:, j]).max())
                          for j in range(6)))
        variants[prec] = {"ms_per_launch": vms, "speedup_vs_fp64_plan": ms / vms,
                          "max_rel_err_element0_of_every_set": err}
        bv.close()
    for P, _, _ in items:
        stp.stp_set_precision(P.handle, "fp64")
    out = {"workload": "64 element sets, orders 3-11 (N=4..12), "
                       f"64-{args.batched_emax} elements each "
                       "(log-uniform, seed 1003), one persistent launch per shape from a CUDA graph",
           "sets": len(recipe), "elements": elems, "ms_per_launch": ms,
           "elements_per_s": elems / (ms / 1e3), "tflops_algorithmic": flops / (ms / 1e3) / 1e12,
           "frac_fp64_peak": flops / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
           "plan_seconds_incl_autotune": plan_s, **b.info(),
           "variants_graph_of_launches": variants,
           "autotune": {str(n): {"variant": t["variant"],
                                 "us_per_element": [round(u, 4) for u in t["us_variants"]]}
                        for n, t in sorted(tuned.items())}}
    b.close()
    for P, _, _ in items:
        P.close()
    return out


def copy_bound(torch, dev, host_in, host_out, reps=3):
    """The host-link side of the e2e roofline: the step's own pinned buffers
    copied in (host to device) and out (device to host), each direction
    alone and both at once on two streams (best of `reps`)."""
    d_in = [torch.empty_like(t, device=dev) for t in host_in]
    d_out = [torch.empty_like(t, device=dev) for t in host_out]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def h2d():
        with torch.cuda.stream(s_in):
            for d, h in zip(d_in, host_in):
                d.copy_(h, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s_out):
            for h, d in zip(host_out, d_out):
                h.copy_(d, non_blocking=True)

    def best(fns):
        t = float("inf")
        for _ in range(reps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for f in fns:
                f()
            torch.cuda.synchronize(dev)
            t = min(t, time.perf_counter() - t0)
        return t

    b_in = sum(t.numel() * t.element_size() for t in host_in)
    b_out = sum(t.numel() * t.element_size() for t in host_out)
    t_in, t_out, t_both = best([h2d]), best([d2h]), best([h2d, d2h])
    del d_in, d_out
    return {"h2d_gbs": b_in / t_in / 1e9, "d2h_gbs": b_out / t_out / 1e9,
            "both_ms": t_both * 1e3, "note": "pinned copies of one step's inputs and outputs; "
            "the e2e step cannot beat max(kernel time, both_ms)"}


def served_measurement(stp, torch, args):
    """The served workload: 256 simulations (orders 3-9, N=4..10, element
    counts log-uniform in [64, args.served_emax], seed 1005, state and
    material generated on the GPU), a device pool of args.served_budget_gb,
    Poisson arrivals at args.served_rate req/s (seed 1006), each picking a
    simulation uniformly. args.served_warmup requests are replayed first; then
    args.served_requests are timed. Latency = completion seen by the scheduler
    minus arrival. A second trace (args.served_sub_requests, seed 1007) then
    runs on the same server at 0.7x the throughput the first one measured, so
    that its latency is service time rather than queueing."""
    from paper_2003_12787_gb300.inputs import elastic_problem, served_arrivals, served_recipe
    recipe = served_recipe(e_max=args.served_emax)
    budget = int(args.served_budget_gb * (1 << 30))
    srv = stp.Server(budget, slots=args.served_slots)
    preds = []
    for r in recipe:
        prob = elastic_problem(r["N"], grid=r["grid"], E=r["E"], h=r["h"],
                               seed_material=r["seed_material"], seed_waves=r["seed_waves"],
                               device="cuda")
        P = stp.Predictor(r["N"] - 1, prob.h, prob.dt)
        srv.add_sim(P, prob.q, prob.params)
        preds.append(P)
        del prob
    E = np.array([r["E"] for r in recipe])

    def timed_trace(rate, n_w, n_m, seed):
        t, ids = served_arrivals(n_w + n_m, rate=rate, n_sims=len(recipe), seed=seed)
        if n_w:
            srv.run_trace(t[:n_w] - t[0], ids[:n_w])
        before = srv.stats()
        t_m = t[n_w:] - t[n_w]
        lat, wall = srv.run_trace(t_m, ids[n_w:])
        after = srv.stats()
        launches = after["launches"] - before["launches"]
        return {"rate_req_s": rate, "requests": n_m, "warmup_requests": n_w,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "wall_s": wall,
                "throughput_req_s": n_m / wall,
                "element_updates_per_s": int(E[ids[n_w:]].sum()) / wall,
                "offered_req_s": n_m / float(t_m[-1]) if n_m > 1 else None,
                "launches": launches, "mean_batch": n_m / max(1, launches),
                "admissions": after["admissions"] - before["admissions"],
                "evictions": after["evictions"] - before["evictions"],
                "pool_peak_gb": after["pool_bytes_peak"] / 2 ** 30,
                "launch_device_s": (after["kernel_us"] - before["kernel_us"]) / 1e6}

    main = timed_trace(args.served_rate, args.served_warmup, args.served_requests, 1006)
    out = {"workload": "256 simulations, orders 3-9 (N=4..10), "
                       f"64-{args.served_emax} elements each (log-uniform, seed 1005), "
                       f"Poisson {args.served_rate:g} req/s (seed 1006), one FP64 STP step per request",
           "hbm_budget_gb": args.served_budget_gb, "slots": args.served_slots,
           "total_state_gb": float(sum(8 * r["E"] * (21 * r["N"] ** 3 + 54 * r["N"] ** 2)
                                       for r in recipe) / 2 ** 30), **main}
    if args.served_sub_requests > 0:
        # the same server below its measured capacity, so that latency is
        # service time rather than queueing (arrivals seed 1007), with the
        # default resident-first order and then with FIFO on the same trace
        sub_rate = 0.7 * main["throughput_req_s"]
        out["below_capacity"] = timed_trace(sub_rate, 0, args.served_sub_requests, 1007)
        out["below_capacity"]["policy"] = "resident first, age bound 0.05 s"
        srv.set_policy(0)
        out["below_capacity_fifo"] = timed_trace(sub_rate, 0, args.served_sub_requests, 1007)
        out["below_capacity_fifo"]["policy"] = "FIFO"
        srv.set_policy(1, 0.05)
    if not args.no_served_ff:
        # the same trace with every simulation's handle switched to float-float
        # (FP64-class results, one launch per simulation instead of the
        # persistent FP64 batch)
        for P in preds:
            stp.stp_set_precision(P.handle, "ff")
        out["float_float"] = timed_trace(args.served_rate, args.served_warmup,
                                         args.served_requests, 1006)
    srv.close()
    for P in preds:
        P.close()
    return out


def served_cfg5_measurement(stp, torch, args):
    """The served workload at its stated sizes: 256 simulations, orders 3-9,
    64-32768 elements each (log-uniform, seed 1005), state and material
    generated on the GPU and added from device buffers (they start resident;
    pinned host copies would be made only on eviction), a pool of
    args.cfg5_budget_gb, Poisson arrivals at args.served_rate req/s (seed
    1006): far above the FP64 capacity (about 8.7 GFLOP per request), so the
    latency of the over-capacity trace is queueing, reported as measured. A
    second trace at 0.7x the measured throughput (seed 1007) gives the service
    latency."""
    from paper_2003_12787_gb300.inputs import elastic_problem, served_arrivals, served_recipe
    recipe = served_recipe(e_max=32768)
    budget = int(args.cfg5_budget_gb * 1e9)
    srv = stp.Server(budget, slots=args.served_slots)
    preds = []
    for r in recipe:
        prob = elastic_problem(r["N"], grid=r["grid"], E=r["E"], h=r["h"],
                               seed_material=r["seed_material"], seed_waves=r["seed_waves"],
                               device="cuda")
        P = stp.Predictor(r["N"] - 1, prob.h, prob.dt)
        srv.add_sim(P, prob.q, prob.params)
        preds.append(P)
        del prob
    torch.cuda.empty_cache()
    E = np.array([r["E"] for r in recipe])
    flops = np.array([r["E"] * flops_per_element(r["N"]) for r in recipe], dtype=np.float64)

    def trace(rate, n, seed):
        t, ids = served_arrivals(n, rate=rate, n_sims=len(recipe), seed=seed)
        before = srv.stats()
        lat, wall = srv.run_trace(t - t[0], ids)
        after = srv.stats()
        launches = after["launches"] - before["launches"]
        return {"rate_req_s": rate, "requests": n,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "wall_s": wall,
                "throughput_req_s": n / wall,
                "element_updates_per_s": int(E[ids].sum()) / wall,
                "tflops_algorithmic": float(flops[ids].sum()) / wall / 1e12,
                "launches": launches, "mean_batch": n / max(1, launches),
                "admissions": after["admissions"] - before["admissions"],
                "evictions": after["evictions"] - before["evictions"],
                "pool_peak_gb": after["pool_bytes_peak"] / 1e9}

    over = trace(args.served_rate, args.cfg5_requests, 1006)
    out = {"workload": "256 simulations, orders 3-9 (N=4..10), 64-32768 elements each "
                       "(log-uniform, seed 1005), one FP64 STP step per request",
           "hbm_budget_gb": args.cfg5_budget_gb,
           "total_footprint_gb": float(sum(8 * r["E"] * (21 * r["N"] ** 3 + 54 * r["N"] ** 2
                                                         + 9 * r["N"] ** 3) for r in recipe) / 1e9),
           "mean_gflop_per_request": float(flops.mean() / 1e9),
           "over_capacity": over}
    if args.cfg5_sub_requests > 0:
        out["below_capacity"] = trace(0.7 * over["throughput_req_s"], args.cfg5_sub_requests, 1007)
    srv.close()
    for P in preds:
        P.close()
    torch.cuda.empty_cache()
    return out


def corrector_fp64_ops_per_node(N: int) -> int:
    """FP64 instructions the corrector issues per node: 18 derivative chains of
    N DFMA (elastic sparsity), 12 for the elastic update, 54 for the lift of
    the six face fluctuations (9 quantities x 6 faces) and 9 for q + update."""
    return 18 * N + 12 + 54 + 9


def ader_measurement(stp, torch, args):
    """Full ADER-DG steps (predictor + corrector) on the periodic order-7
    workload: the corrector alone, the predictor alone and whole steps through
    stp_ader_step; sampled elements checked against the oracle."""
    import oracle
    from paper_2003_12787_gb300.inputs import ader_order7_case
    prob = ader_order7_case(device="cuda")
    E, N, grid = prob.E, prob.N, prob.grid
    P = stp.Predictor(N - 1, prob.h, prob.dt)
    s = torch.cuda.current_stream()
    qd = prob.q.clone()
    fp = P.face_params(prob.params)
    avg, faces = P.empty_outputs(E)
    out = torch.empty_like(qd)

    def timed(fn, reps):
        for _ in range(3):
            fn()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(s)
        for _ in range(reps):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    P.predict(prob.q, prob.params, out=(avg, faces))
    pred_ms = timed(lambda: P.predict(prob.q, prob.params, out=(avg, faces)), 5)
    corr_ms = timed(lambda: P.correct(grid, prob.q, prob.params, fp, avg, faces, out=out), 10)
    fp_ms = timed(lambda: P.face_params(prob.params), 5)
    steps = 5
    qd.copy_(prob.q)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    P.ader_steps(grid, qd, prob.params, fp, steps, work=(avg, faces))
    b.record(s)
    torch.cuda.synchronize()
    step_ms = a.elapsed_time(b) / steps
    # parity: one step from the initial state, sampled elements vs the oracle
    qd.copy_(prob.q)
    P.ader_steps(grid, qd, prob.params, fp, 1, work=(avg, faces))
    torch.cuda.synchronize()
    q, pa = prob.q.cpu().numpy(), prob.params.cpu().numpy()
    got = qd.cpu().numpy()
    gx, gy, gz = grid
    err = 0.0
    for e in (0, E // 2 + 17, E - 1):
        ex, ey, ez = e % gx, (e // gx) % gy, e // (gx * gy)
        idx = [((ez + dz) % gz * gy + (ey + dy) % gy) * gx + (ex + dx) % gx
               for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        ref = oracle.ader_steps(q[idx], pa[idx], (3, 3, 3), prob.h, prob.dt, 1)[13]
        err = max(err, float(np.abs(got[e] - ref).max() / np.abs(ref).max()))
    ops = corrector_fp64_ops_per_node(N) * N ** 3
    P.close()
    return {"workload": "order-7 (N=8) full ADER-DG step (predictor + corrector, Rusanov flux), "
                        "periodic 32^3 grid of side 1/32, element-wise material",
            "elements": E, "predictor_ms": pred_ms, "corrector_ms": corr_ms,
            "face_params_ms_once_per_mesh": fp_ms, "step_ms": step_ms,
            "steps_timed": steps, "element_steps_per_s": E / (step_ms / 1e3),
            "corrector_share_of_step": corr_ms / step_ms,
            "corrector_fp64_ops_per_element": ops,
            "corrector_fp64_pipe_frac_est": E * ops / (corr_ms / 1e3) /
            (FP64_PEAK_TFLOPS * 1e12 / 2),
            # algorithmic bytes: q, avg, params, q_out, faces and face_params once each
            "corrector_hbm_gbs": E * 8 * (30 * N ** 3 + 54 * N ** 2 + 18 * N ** 2) /
            (corr_ms / 1e3) / 1e9,
            "max_rel_err_sampled_one_step": err}


def compact_summary(line):
    """The secondary figures in a few hundred characters, placed last in the
    line: speed-up and error per arithmetic variant at order 9, the batched
    plan's FP64 fraction, the served trace's rate and latency, the full
    ADER-DG step and the small-case latency."""
    def r(x, n=4):
        return None if x is None else float(f"{x:.{n}g}")
    out = {"fp64_frac": r(line["roofline"]["frac"]),
           "fp64_pipe_frac": r(line["roofline"].get("fp64_pipe_frac"))}
    mixed = line.get("mixed")
    if mixed:
        out["order9_speedup_err"] = {k: [r(v["speedup_vs_fp64"], 3), r(v["max_rel_err"], 2)]
                                     for k, v in mixed["variants"].items()}
    b = line.get("batched")
    if b:
        out["batched"] = {"ms": r(b["ms_per_launch"]), "fp64_frac": r(b["frac_fp64_peak"])}
    sv = line.get("served")
    if sv:
        out["served"] = {"req_s": r(sv["throughput_req_s"]), "p50_ms": r(sv["p50_ms"]),
                         "p99_ms": r(sv["p99_ms"])}
        bc = sv.get("below_capacity")
        if bc:
            out["served"]["below_capacity"] = [r(bc["throughput_req_s"]), r(bc["p50_ms"]),
                                               r(bc["p99_ms"])]
        ff = sv.get("float_float")
        if ff:
            out["served"]["ff"] = [r(ff["throughput_req_s"]), r(ff["p50_ms"]), r(ff["p99_ms"])]
        bf = sv.get("below_capacity_fifo")
        if bf:
            out["served"]["below_capacity_fifo"] = [r(bf["throughput_req_s"]), r(bf["p50_ms"]),
                                                    r(bf["p99_ms"])]
    c5 = line.get("served_cfg5")
    if c5:
        o = c5["over_capacity"]
        out["served_cfg5"] = {"req_s": r(o["throughput_req_s"]), "p50_ms": r(o["p50_ms"]),
                              "p99_ms": r(o["p99_ms"]), "tflops": r(o["tflops_algorithmic"])}
        b = c5.get("below_capacity")
        if b:
            out["served_cfg5"]["below_capacity"] = [r(b["throughput_req_s"]), r(b["p50_ms"]),
                                                    r(b["p99_ms"])]
    a = line.get("ader_step")
    if a:
        out["ader_step"] = {"step_ms": r(a["step_ms"]), "corrector_ms": r(a["corrector_ms"]),
                            "err": r(a["max_rel_err_sampled_one_step"], 2)}
    sc = line.get("small_case")
    if sc:
        out["small_case_us_p50_p99"] = [r(sc["device_us"]["p50"]), r(sc["device_us"]["p99"])]
    return out


def run_gpu(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    import paper_2003_12787_gb300 as stp
    from paper_2003_12787_gb300.inputs import elastic_problem

    N, grid, h, desc = WORKLOADS[args.workload]
    curv = args.geometry == "curvilinear"
    if curv:
        from paper_2003_12787_gb300.inputs import curvilinear_problem
        if args.precision not in ("fp64", "ff", "fp32"):
            raise SystemExit("curvilinear elements run in FP64, float-float or FP32 only")
        prob = curvilinear_problem(N, grid=grid, h=h, seed_material=1001 + 16 * rank,
                                   seed_waves=1002 + 16 * rank, device="cuda")
        desc = desc.replace("elastic STP,", "elastic STP on curvilinear elements (smooth map "
                                            "of amplitude 0.2),")
    else:
        prob = elastic_problem(N, grid=grid, h=h, seed_material=1001 + 16 * rank,
                               seed_waves=1002 + 16 * rank, device="cuda")
    metric = prob.metric  # None on Cartesian cubes
    E = prob.E
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    P = stp.Predictor(N - 1, prob.h, prob.dt, precision=args.precision)
    avg, faces = P.empty_outputs(E, device=dev)

    fp64_probe = stp.stp_measure_fp64_peak(stream)
    dmma_probe = stp.stp_measure_fp64_peak_kind("dmma", stream)

    for _ in range(args.warmup):
        P.predict(prob.q, prob.params, out=(avg, faces), stream=stream, metric=metric)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()

    sampler = ClockSampler(dev.index) if rank == 0 else None
    if sampler:
        sampler.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for i in range(args.steps):
        starts[i].record(stream)
        P.predict(prob.q, prob.params, out=(avg, faces), stream=stream, metric=metric)
        ends[i].record(stream)
    t_all1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    total_ms = t_all0.elapsed_time(t_all1)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms_max = max_over_ranks(total_ms, world, dev)
    value = E * args.steps * world / (total_ms_max / 1e3)

    # spot parity of this run's outputs against the oracle (a few elements)
    parity = None
    if rank == 0:
        import oracle
        idx = torch.tensor([0, E // 3, E - 1], device=dev)
        if curv:
            a_ref, f_ref = oracle.stp_curvilinear(prob.q[idx].cpu().numpy(),
                                                  prob.params[idx].cpu().numpy(),
                                                  metric[idx].cpu().numpy(), prob.dt)
        else:
            a_ref, f_ref = oracle.stp(prob.q[idx].cpu().numpy(), prob.params[idx].cpu().numpy(),
                                      prob.h, prob.dt)
        a = avg[idx].cpu().numpy()
        f = faces[idx].cpu().numpy()
        parity = max(float(np.abs(a - a_ref).max() / np.abs(a_ref).max()),
                     float(np.abs(f - f_ref).max() / np.abs(f_ref).max()))

    # end to end through the host-buffer entry point (pinned memory)
    e2e = None
    if not args.no_e2e:
        qh = prob.q.cpu().pin_memory()
        ph = prob.params.cpu().pin_memory()
        mh = metric.cpu().pin_memory() if curv else None
        ah, fh = P.empty_outputs(E, device="cpu", pin_memory=True)
        P.predict_host(qh, ph, out=(ah, fh), metric=mh)  # warm-up: allocates staging buffers
        barrier(world)
        t0 = time.perf_counter()
        ke = max(1, min(args.steps, 5))
        call_ms = []
        for _ in range(ke):
            tc = time.perf_counter()
            P.predict_host(qh, ph, out=(ah, fh), metric=mh)
            call_ms.append(round((time.perf_counter() - tc) * 1e3, 2))
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": E * ke * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(qh.numel() * 8 + ph.numel() * 8 +
                                         (mh.numel() * 8 if curv else 0)),
               "d2h_bytes_per_step": int(ah.numel() * 8 + fh.numel() * 8),
               "steps": ke, "ms_per_call": call_ms}
        if not np.array_equal(ah[:4].numpy(), avg[:4].cpu().numpy()):
            e2e["mismatch_vs_device_path"] = True
        e2e["copy_bound"] = copy_bound(torch, dev, [qh, ph] + ([mh] if curv else []), [ah, fh])

    extras = rank == 0 and world == 1 and not curv
    mixed = variants7 = None
    if extras and not args.no_mixed:
        mixed = mixed_comparison(stp, torch, args)
        variants7 = mixed_comparison(stp, torch, args, workload=args.workload,
                                     precisions=("fp64", "ff", "fp32"))
    curvilinear = None
    if extras and not args.no_curvilinear and args.workload == "order7" \
            and args.precision == "fp64":
        curvilinear = curvilinear_measurement(stp, torch, args, statistics.mean(step_ms))
    small = None
    if extras and args.small_launches > 0:
        small = small_case_latency(stp, torch, args)
    batched = None
    if extras and not args.no_batched:
        batched = batched_measurement(stp, torch, args)
    served = None
    if extras and not args.no_served:
        served = served_measurement(stp, torch, args)
    served_cfg5 = None
    if extras and not args.no_served and args.cfg5_requests > 0:
        served_cfg5 = served_cfg5_measurement(stp, torch, args)
    ader = None
    if extras and not args.no_ader:
        ader = ader_measurement(stp, torch, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        qn = prob.q.cpu().numpy()
        pn = prob.params.cpu().numpy()
        mn = metric.cpu().numpy() if curv else None
        done, spent, cores = oracle_baseline(qn, pn, prob.h, prob.dt, args.cpu_budget, E, mn)
        cpu = {"value": done / spent, "unit": UNIT, "cores": cores, "cpu": cpu_model(),
               "kind": "oracle",
               "sample": f"first {done} of {E} elements of the same workload, "
                         f"{spent:.1f} s wall on {cores} OpenMP threads"}

    if rank == 0:
        mean_step_s = statistics.mean(step_ms) / 1e3
        fpe = flops_per_element_curvilinear(N) if curv else flops_per_element(N)
        bpe = 8 * (30 * N ** 3 + 54 * N ** 2) if curv else bytes_per_element(N)
        achieved = E * fpe / mean_step_s / 1e12
        srt = sorted(step_ms)
        p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
        traffic = None if curv else traffic_from_profile(args.workload)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32+ff32", "ff": "ff32"}.get(args.precision, f"{args.precision}+f32+f64"),
            "data": "synthetic",
            "config": {"workload": desc, "N": N, "order": N - 1, "elements": E,
                       "elements_per_gpu": E, "dt": prob.dt, "dx": prob.h,
                       "l2": "inputs larger than L2: %.2f GB read + %.2f GB written per step"
                             % (E * 8 * (21 if curv else 12) * N ** 3 / 1e9,
                                E * 8 * (9 * N ** 3 + 54 * N ** 2) / 1e9),
                       "parallelism": f"dp{world} (element partitions, no collective)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                         "traffic": traffic,
                         "peak_kind": "derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz",
                         "fp64_probe_tflops": fp64_probe / 1e3,
                         "dmma_probe_tflops": dmma_probe / 1e3,
                         "fp64_pipe_frac": None if curv else fp64_pipe_fraction(
                             args.workload, mean_step_s * 1e3, (clocks or {}).get("sm_mhz")),
                         "traffic_source": "stored ncu record of this kernel source (4096-element "
                                           "capture scaled by elements), not measured in this run",
                         "frac_of_probe": achieved / (fp64_probe / 1e3),
                         "flops_per_element": fpe,
                         "flops_per_element_dense_count": None if curv else flops_per_element_dense(N),
                         "tflops_dense_count": None if curv else
                         E * flops_per_element_dense(N) / mean_step_s / 1e12,
                         "hbm_gbs": E * bpe / mean_step_s / 1e9},
            "latency_ms": {"p50": statistics.median(step_ms), "p99": p99,
                           "min": min(step_ms), "max": max(step_ms)},
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "mixed": mixed, "variants_same_workload": variants7,
            "small_case": small, "batched": batched, "served": served, "served_cfg5": served_cfg5,
            "curvilinear": curvilinear, "ader_step": ader,
            "gpu_launches": args.steps, "parity_max_rel_sampled": parity,
            "paper_context": {
                "figure": "22.5 % of available FP64 performance",
                "kernel": "AoSoA SplitCK STP, N = 11, elastic LOH1 on a curvilinear mesh (m = 21)",
                "cpu": "8 cores of an Intel Xeon Platinum 8174 at 1.9 GHz under AVX-512, "
                       "60.8 GFLOP/s per core available",
                "this_run_frac_of_fp64_peak": achieved / FP64_PEAK_TFLOPS},
        }
        line["summary"] = compact_summary(line)  # last key: survives a cut-off tail
        print(json.dumps(line), flush=True)
    P.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2003_12787_gb300.inputs import elastic_problem
    N, grid, h, desc = WORKLOADS[args.workload]
    prob = elastic_problem(N, grid=grid, h=h)
    q = prob.q.numpy()
    p = prob.params.numpy()
    sample = min(prob.E, args.reference_sample)
    qs, ps = np.ascontiguousarray(q[:sample]), np.ascontiguousarray(p[:sample])
    for _ in range(args.warmup):
        oracle.stp(qs, ps, prob.h, prob.dt)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.stp(qs, ps, prob.h, prob.dt)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sample * args.steps / total
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "N": N, "order": N - 1, "elements": prob.E,
                   "sample_elements_per_step": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": cpu_model(),
                         "kind": "oracle",
                         "sample": f"first {sample} of {prob.E} elements per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def build_parser():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="order7")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the precision-variant comparisons (order-9 workload and the timed workload)")
    ap.add_argument("--mixed-steps", type=int, default=5)
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched 64-set workload")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batched-emax", type=int, default=16384,
                    help="largest set of the batched workload (smaller for profiler captures)")
    ap.add_argument("--no-served", action="store_true", help="skip the served workload")
    ap.add_argument("--no-ader", action="store_true",
                    help="skip the full ADER-DG step (predictor + corrector) measurement")
    ap.add_argument("--no-served-ff", action="store_true",
                    help="skip the float-float run of the served trace")
    ap.add_argument("--no-curvilinear", action="store_true",
                    help="skip the curvilinear order-7 measurement")
    ap.add_argument("--geometry", choices=["cartesian", "curvilinear"], default="cartesian",
                    help="time the main workload on Cartesian cubes (default) or on "
                         "curvilinear elements (fp64, ff or fp32; no extras)")
    ap.add_argument("--small-launches", type=int, default=50,
                    help="timed launches of the order-3 latency measurement (0: skip)")
    ap.add_argument("--served-rate", type=float, default=2000.0)
    ap.add_argument("--served-requests", type=int, default=20000)
    ap.add_argument("--served-warmup", type=int, default=1000)
    ap.add_argument("--served-sub-requests", type=int, default=5000,
                    help="requests of the second trace at 0.7x the measured capacity (0: skip)")
    ap.add_argument("--served-emax", type=int, default=2048)
    ap.add_argument("--served-budget-gb", type=float, default=2.0)
    ap.add_argument("--served-slots", type=int, default=3)
    ap.add_argument("--cfg5-requests", type=int, default=1200,
                    help="requests of the full-size served trace (0 skips it)")
    ap.add_argument("--cfg5-sub-requests", type=int, default=300,
                    help="requests of its below-capacity trace")
    ap.add_argument("--cfg5-budget-gb", type=float, default=160.0,
                    help="HBM pool of the full-size served trace (GB)")
    ap.add_argument("--precision", default="fp64",
                    choices=list(PRECISIONS_ALL),
                    help="arithmetic of the timed workload (default fp64)")
    ap.add_argument("--cpu-budget", type=float, default=10.0,
                    help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--reference-sample", type=int, default=1024,
                    help="elements per step of the reference arm")
    return ap


def main():
    args = build_parser().parse_args()
    if args.warmup < 3 and args.impl == "gpu":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
