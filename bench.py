#!/usr/bin/env python
"""Benchmark: IIM solves/s of the 1024^2 star-interface problem on GB300.

One *step* is one complete pass of the solver path over one input: device
set-up from the geometry (control points, curvature check, least-squares fits,
correction records, Shortley-Weller levels, coarse LU), the data term
b = f - L_Gamma u_Gamma, and the FP64 FGMRES(10) solve preconditioned by one
FP32 SW-multigrid V-cycle down to relative residual 1e-10.  Every step solves a
different manufactured problem on the same geometry (seeded), with its inputs
resident in HBM before the timed region; L2 is flushed between steps.

Lines printed (rank 0): one JSON object.  ``--impl reference`` times the CPU
oracle instead (rank 0 only).  Multi-GPU: each rank solves its own problems
(weak scaling, no data-path collective); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IIM solves/s to rel. resid 1e-10 (FP32-MG form)"
WORKLOAD = "star_interface_1024_o6"
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-roofline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="host-driven FGMRES loop (for kernel-level profiling)")
    ap.add_argument("--batch", type=int, default=8, help="independent problems solved concurrently per step")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms, world):
    """The slowest rank's timed region (ms); a collective on the timing only."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, max_ms):
    """Units per second over all ranks (weak scaling: every rank solves its own problems)."""
    return world * units_per_rank / (max_ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": HBM_FALLBACK_GBS, "sm_max_mhz": 2070.0}, "fallback"


# FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA/clk x 2 flop x f_max
def fp64_peak_tflops(sm_max_mhz):
    return 152 * 2 * 2 * sm_max_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"iim_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(P, steps, n, rank, index=0, batch=1):
    """Per-step data at the problem's own control points (fixed geometry per problem)."""
    import numpy as np
    import torch

    import workloads as W
    xc, nc = P.control_points()
    xc, nc = xc.cpu().numpy(), nc.cpu().numpy()
    phase = P.phase().cpu().numpy().astype(bool)
    X = W.node_coords(n, 2)
    plus = W.from_flat(phase, n, 2)
    dev_in, host_in, specs = [], [], []
    for s in range(steps):
        spec = W.star_interface_variant(n, s + 1000 * (rank * batch + index), angle=star_angle(index, batch))
        f = W.to_flat(W.source_term(spec, X, plus))
        g, j0, j1 = W.boundary_data(spec, xc, nc)
        box = W.box_data(spec)
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (f, j0, j1, box)]
        dev_in.append([h.to("cuda") for h in host])
        host_in.append(host)
        specs.append(spec)
    return dev_in, host_in, specs


def star_angle(index, batch):
    """Problem i of a batch solves the star rotated by 2 pi i / (5 batch)."""
    import math
    return 2 * math.pi * index / (5 * max(batch, 1))


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as ge
    import paper_2503_22455_gb300 as iim
    try:
        iim.load()
    except ImportError:
        ge.build()
        iim.load()
    import workloads as W

    n, B = args.n, max(1, args.batch)
    K, Wm = args.steps, args.warmup
    main = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(B)]
    specs0 = [W.star_interface_1024(n, phase=star_angle(i, B)) for i in range(B)]
    opts = iim.default_options(tol=1e-10, mg_precision=iim.MG_FP32, use_graph=0 if args.no_graph else 1)
    probs = [iim.Problem(iim.desc_from_spec(sp), opts, st) for sp, st in zip(specs0, streams)]
    inputs = [make_inputs(P, Wm + K, n, rank, i, B) for i, P in enumerate(probs)]
    xs = [torch.zeros(P.N, dtype=torch.float64, device="cuda") for P in probs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2 (129 MB)
    torch.cuda.synchronize()

    def step(s, problems, xvec):
        """Set-up + data + solve of every problem of the batch, concurrently on their streams."""
        l0 = iim.launch_count()
        start = torch.cuda.Event()
        start.record(main)
        for i, P in enumerate(problems):
            st = streams[i]
            st.wait_event(start)
            with torch.cuda.stream(st):
                P.setup()
                f, j0, j1, box = inputs[i][0][s]
                P.set_data(f, None, j0, j1, box)
                xvec[i].zero_()
        if len(problems) == 1 and args.no_graph:
            _, info = problems[0].solve(xvec[0])
            infos = [info]
        else:
            infos, _ = iim.batch_solve(problems, xvec)
        for st in streams[:len(problems)]:
            main.wait_stream(st)
        kern = iim.launch_count() - l0 - sum(1 for _ in infos) + sum(inf.kernels for inf in infos)
        return infos, kern

    for s in range(Wm):
        step(s, probs, xs)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    iters, launches = [], 0
    torch.cuda.nvtx.range_push("timed")
    for k in range(K):
        flush.zero_()
        ev[k][0].record(main)
        infos, nl = step(Wm + k, probs, xs)
        ev[k][1].record(main)
        launches += nl
        for inf in infos:
            iters.append(inf.iters)
            if not inf.converged:
                raise RuntimeError(f"step {k} did not converge: {inf.as_dict()}")
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    value = whole_job_rate(B * K, world, total_ms)

    # accuracy of the last step of problem 0 against its manufactured solution
    spec = inputs[0][2][Wm + K - 1]
    ph = probs[0].phase().cpu().numpy().astype(bool)
    Xn = W.node_coords(n, 2)
    ex = W.to_flat(np.where(W.from_flat(ph, n, 2), spec.solution.u_plus(Xn), spec.solution.u_minus(Xn)))
    err_exact = float(np.max(np.abs(xs[0].cpu().numpy() - ex)))

    # latency of one solve (batch of one, the same problem)
    lat = []
    for k in range(min(K, 5)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        step(Wm + k, probs[:1], xs[:1])
        b.record(main)
        torch.cuda.synchronize()
        lat.append(a.elapsed_time(b))

    fp64_form = None
    if args.fp64_steps > 0:
        fp64_form = fp64_run(args, iim, torch, specs0, streams, inputs, step, flush, Wm, main)
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(probs, torch, inputs, Wm, K, world, main)
    roof = None if args.no_roofline else roofline(probs[0], iim, torch, main)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, statistics.mean(iters))
    pk, src = peaks()
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "mg_dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "order": 6, "bc": "interface", "box": "dirichlet",
                   "geometry": "star r=0.5+0.1 sin(5 theta), rotated per problem", "tol": 1e-10,
                   "krylov": "FGMRES(10), right", "preconditioner": "SW multigrid V(2,2), fp32",
                   "batch": B, "l2": "flushed between steps", "step": "per problem: setup+data+solve"},
        "latency_ms_single_solve": statistics.median(lat),
        "iters_mean": statistics.mean(iters), "err_vs_exact": err_exact,
        "fp64_form": fp64_form,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk,
        "peaks_source": src,
    }
    if cpu:
        out["cpu_baseline"] = cpu
    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def fp64_run(args, iim, torch, specs0, streams, inputs, step, flush, Wm, main):
    """The all-FP64 form (FP64 multigrid), same batch and inputs."""
    import statistics as st
    opts = iim.default_options(tol=1e-10, mg_precision=iim.MG_FP64)
    probs = [iim.Problem(iim.desc_from_spec(sp), opts, s) for sp, s in zip(specs0, streams)]
    xs = [torch.zeros(P.N, dtype=torch.float64, device="cuda") for P in probs]
    step(0, probs, xs)
    t, it = [], []
    for k in range(args.fp64_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        infos, _ = step(Wm + k, probs, xs)
        b.record(main)
        torch.cuda.synchronize()
        t.append(a.elapsed_time(b))
        it += [inf.iters for inf in infos]
    for P in probs:
        P.close()
    return {"value": len(probs) * 1e3 / st.mean(t), "unit": "solves/s", "iters": st.mean(it)}


def e2e_run(probs, torch, inputs, Wm, K, world, main):
    """End to end through the host-buffer entry point (one host thread per problem):
    H2D of every step's inputs and D2H of x inside the timed region."""
    import concurrent.futures as cf
    xh = [torch.empty(P.N, dtype=torch.float64).pin_memory() for P in probs]

    def one(i, k):
        P = probs[i]
        f, j0, j1, box = inputs[i][1][Wm + k]
        P.setup()
        P.solve_host(f, None, j0, j1, box, x=xh[i])

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=len(probs)) as ex:
        for k in range(K):
            list(ex.map(lambda i: one(i, k), range(len(probs))))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = sum(t.numel() * 8 for t in inputs[0][1][Wm])
    return {"value": world * len(probs) * K / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d * len(probs),
            "d2h_bytes_per_step": probs[0].N * 8 * len(probs)}


def roofline(P, iim, torch, stream):
    """Dominant kernel: the FP64 high-order stencil (bound by the FP64 pipe).

    Algorithmic FP64 work per unknown node: w(2d-1) adds to pair the 2dw
    neighbours by |j|, w multiply-adds and one multiply -> w(2d+1)+1 flop
    (16 for the 2D sixth-order stencil).  Timed live with CUDA events on the
    problem's stream over repeated launches of the same kernel on the solve's
    own vectors.
    """
    import ctypes
    lib = iim.load()
    us = ctypes.c_double()
    reps = 50
    st = lib.iim_kernel_time(P.h, 0, reps, ctypes.byref(us))
    if st != 0:
        return None
    d, w = 2, 3
    flops = (w * (2 * d + 1) + 1) * P.n_unknowns
    achieved = flops / (us.value * 1e-6) / 1e12
    pk, src = peaks()
    peak = fp64_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    return {"kernel": "k_ho_stencil<2,3>", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s (FP64)", "frac": achieved / peak, "traffic": None, "us_per_launch": us.value,
            "peak_note": "152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock"}


def cpu_baseline(n, gpu_iters):
    """The oracle on the host: set-up + one FGMRES(10) cycle, scaled to one full solve."""
    r = oracle_sample(n, gpu_iters)
    return {"value": r["value"], "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": r["sample"]}


def oracle_sample(n, iters_full):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np

    import workloads as W
    from oracle.fgmres import fgmres
    from oracle.problem import OracleProblem
    spec = W.star_interface_variant(n, 0)
    t0 = time.perf_counter()
    O = OracleProblem(spec)
    f, data = O.data()
    _ = O.mg
    b = O.op.rhs(f, data)
    t1 = time.perf_counter()
    fgmres(O.op.apply, O.precondition, b, tol=1e-10, restart=10, max_iter=10)
    t2 = time.perf_counter()
    per_iter = (t2 - t1) / 10
    solve_s = (t1 - t0) + per_iter * iters_full
    return {"value": 1.0 / solve_s, "seconds": t2 - t0,
            "sample": f"oracle set-up + 10 FGMRES iterations of the {n}^2 problem ({t2 - t0:.1f} s), "
                      f"scaled to one solve of {iters_full:.0f} iterations"}


def oracle_full_iters(n):
    """The oracle's own FGMRES iteration count for the workload (one complete solve)."""
    import workloads as W
    from oracle.problem import OracleProblem
    O = OracleProblem(W.star_interface_variant(n, 0))
    f, data = O.data()
    _, info, _ = O.solve(f, data, tol=1e-10)
    return info["iters"]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    iters_full = oracle_full_iters(args.n)            # the first warm-up step is a complete solve
    for _ in range(max(0, args.warmup - 1)):
        oracle_sample(args.n, iters_full)
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_sample(args.n, iters_full)
        vals.append(1.0 / r["value"])
        secs.append(r["seconds"])
    value = args.steps / sum(vals)
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * sum(vals) / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": args.n, "order": 6, "tol": 1e-10},
           "cpu_baseline": {"value": value, "unit": "solves/s", "kind": "oracle", "cores": 1,
                            "sample": f"per step: oracle set-up + 10 FGMRES iterations, scaled to "
                                      f"{iters_full} iterations"},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
