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
# Many problems run on their own streams at once (8 solve graphs, 16 pool streams, up to 256
# requests): more hardware work queues than the default 8 keep independent streams from
# waiting on one another.  A per-process setting, read when CUDA starts.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

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
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="steps of each other solver form (FP64 multigrid, W-cycle, left GMRES); 0: none")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other-configs", dest="other_configs", action="store_false",
                    help="skip the 64^2 circle and 256^3 ellipsoid lines measured beside the headline")
    ap.add_argument("--no-roofline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="host-driven FGMRES loop (for kernel-level profiling)")
    ap.add_argument("--batch", type=int, default=8, help="independent problems solved concurrently per step")
    ap.add_argument("--solver", default="pool", choices=["engine", "pool"],
                    help="engine: the batch advances in lock step through the batched engine; pool: one solve "
                         "graph per problem on a pool of streams")
    ap.add_argument("--workload", default="star1024", choices=["star1024", "batch512", "serve", "ellipsoid256"],
                    help="star1024: the headline line; batch512: 512 mixed 2D problems through the batched "
                         "engine; serve: a Poisson request stream through the request loop; ellipsoid256: "
                         "the 256^3 Neumann ellipsoid in the FP32-MG, BF16-residual-MG and all-FP64 forms")
    ap.add_argument("--count", type=int, default=0, help="problems (batch512) or requests (serve); 0 = default")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--ticks-per-run", type=int, default=4, help="serve: engine ticks between admissions")
    ap.add_argument("--slots", type=int, default=256, help="serve: problems resident at once at most")
    ap.add_argument("--create-threads", type=int, default=16, help="serve: host threads creating requests")
    ap.add_argument("--data-threads", type=int, default=8,
                    help="serve: client threads preparing request data (0: on the loop's thread)")
    ap.add_argument("--serve-deadline", type=float, default=300.0,
                    help="serve: fail (with the requests' states) when requests are outstanding after this many s")
    ap.add_argument("--serve-mode", type=int, default=1, choices=[0, 1],
                    help="serve: 0 batched engine, 1 each request's solve graph on its own stream")
    ap.add_argument("--engines", type=int, default=2,
                    help="batched engines, each on its own stream with a share of the problems")
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


def workload_config(n, batch, solver):
    """The headline workload's config, the same in both arms."""
    return {"workload": WORKLOAD, "n": n, "order": 6, "bc": "interface", "box": "dirichlet",
            "geometry": "star r=0.5+0.1 sin(5 theta), rotated per problem", "tol": 1e-10,
            "krylov": "FGMRES(10), right", "preconditioner": "SW multigrid V(2,2), fp32",
            "batch": batch, "l2": "flushed between steps", "step": "per problem: setup+data+solve",
            "solver": solver}


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


def _boundary_inputs(P, spec):
    """Device inputs of a boundary problem at its own control points: f on the device
    (source_term_device), control-point and box data from the host."""
    import numpy as np
    import torch

    import workloads as W
    xc, nc = P.control_points()
    g, _, _ = W.boundary_data(spec, xc.cpu().numpy(), nc.cpu().numpy())
    f = W.source_term_device(spec, P.phase())
    box = W.box_data(spec)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    return f, dev(g), (dev(box) if box.size else None)


def run_batch(args):
    """512 mixed 2D problems (50% interior Dirichlet, 50% exterior Neumann with a Dirichlet
    box, (4,5)/(6,7), ellipses and 5-7 lobe stars, n in 64..512) per step: device set-up,
    data and solve of all of them through the batched engine (persistent kernels, one
    graph launch), next to the same problems through per-problem graphs on a stream pool."""
    import torch

    import paper_2503_22455_gb300 as iim
    import workloads as W
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _load_lib(iim)
    count = args.count or 512
    K, Wm = args.steps, args.warmup
    specs = W.batch_specs(count, seed=2503 + 7919 * rank)
    main = torch.cuda.current_stream()
    pool = [torch.cuda.Stream() for _ in range(16)]
    opts = iim.default_options(tol=1e-10, mg_precision=iim.MG_FP32, use_graph=0 if args.no_graph else 1)
    probs = [iim.Problem(iim.desc_from_spec(sp), opts, pool[i % len(pool)]) for i, sp in enumerate(specs)]
    inputs = []
    for P, sp in zip(probs, specs):
        with torch.cuda.stream(P.stream):
            inputs.append(_boundary_inputs(P, sp))
    torch.cuda.synchronize()
    xs = [torch.zeros(P.N, dtype=torch.float64, device="cuda") for P in probs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ne = max(1, args.engines)
    eng_streams = [main] + [torch.cuda.Stream() for _ in range(ne - 1)]
    engines = [iim.Engine(opts, max_slots=(count + ne - 1) // ne, stream=st) for st in eng_streams]
    E = engines[0]
    tuned = {"done": False}

    def prepare():
        start = torch.cuda.Event()
        start.record(main)
        for P, (f, g, box) in zip(probs, inputs):
            P.stream.wait_event(start)
            with torch.cuda.stream(P.stream):
                P.setup()
                P.set_data(f, g, None, None, box)

    split = []

    def step_engine():
        l0 = iim.launch_count()
        t0 = [e.stats()[1] for e in engines]
        prepare()
        for st in pool:
            main.wait_stream(st)
        mid = torch.cuda.Event(enable_timing=True)
        mid.record(main)
        for st in eng_streams[1:]:
            st.wait_event(mid)
        slots = [engines[i % ne].admit(P) for i, P in enumerate(probs)]
        if not tuned["done"]:
            tuned["ms"] = [e.autotune(reps=3) for e in engines]
            tuned["done"] = True
        for e in engines:
            e.run()
        for e in engines:
            e.poll(wait=True)
        infos = [engines[i % ne].release(sl, x) for i, (sl, x) in enumerate(zip(slots, xs))]
        for st in eng_streams[1:]:
            main.wait_stream(st)
        launches = iim.launch_count() - l0 - ne
        nt = 0
        for e, a in zip(engines, t0):
            kpt, t1 = e.stats()
            launches += kpt * (t1 - a)
            nt = max(nt, t1 - a)
        split.append(mid)
        return infos, nt, launches

    def step_pool():
        prepare()
        for st in pool:
            main.wait_stream(st)
        infos, _ = iim.batch_solve(probs, xs)
        return infos

    for _ in range(Wm):
        step_engine()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    iters, ticks, launches = [], [], 0
    split.clear()
    torch.cuda.nvtx.range_push("timed")
    for k in range(K):
        flush.zero_()
        ev[k][0].record(main)
        infos, nt, nl = step_engine()
        ev[k][1].record(main)
        ticks.append(nt)
        launches += nl
        for inf in infos:
            if not inf.converged:
                raise RuntimeError(f"batch step {k}: {inf.as_dict()}")
            iters.append(inf.iters)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), world)
    value = whole_job_rate(count * K, world, total_ms)
    setup_ms = statistics.mean(ev[k][0].elapsed_time(split[k]) for k in range(K))
    # the same steps through per-problem graphs on a stream pool
    step_pool()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pool_ms = []
    for k in range(min(K, 3)):
        flush.zero_()
        a.record(main)
        step_pool()
        b.record(main)
        torch.cuda.synchronize()
        pool_ms.append(a.elapsed_time(b))
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "mg_dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch{count}_mixed_2d", "problems_per_step": count, "n": "64..512 step 32",
                   "mix": "50% interior Dirichlet / 50% exterior Neumann + Dirichlet box; 50% (4,5) / 50% (6,7); "
                          "ellipses and 5-7 lobe stars", "tol": 1e-10, "l2": "flushed between steps",
                   "step": "per problem: setup+data+solve; solves through the batched engine"},
        "iters_mean": statistics.mean(iters), "iters_max": max(iters), "ticks_per_step": statistics.mean(ticks),
        "setup_data_ms_per_step": setup_ms, "engine_ms_per_step": total_ms / K - setup_ms,
        "engines": ne, "kernels_per_tick": E.stats()[0], "autotune_vcycle_ms": tuned.get("ms"),
        "tile_shapes": E.shapes(),
        "stream_pool_solves_per_s": count * 1e3 / statistics.mean(pool_ms),
        "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out))
    for e in engines:
        e.close()


def serve_run(iim, torch, count, rate, seed, slots=256, ticks_per_run=4, mode=1, create_threads=16,
              deadline_s=300.0, note=None, data_threads=8):
    """A Poisson request stream (mean rate ``rate``/s, ``count`` requests, seeded): 2D n
    128..1024 (stars, ellipses), 3D n 64..192 (ellipsoids, perturbed spheres), interior
    Dirichlet / exterior Neumann, admitted by a budget of 60% of free device memory into
    the request loop; p50/p99 latency from submission to the solution on the host, and
    completed solves per second."""
    import numpy as np

    import workloads as W
    trace = W.serving_trace(count=count, rate=rate, seed=seed)
    opts = iim.default_options(tol=1e-10, mg_precision=iim.MG_FP32)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.6 * free)

    def set_data(view, spec):
        f, g, box = _boundary_inputs(view, spec)
        view.set_data(f, g, None, None, box)

    # warm-up: a few requests through a separate server (library, kernels, allocator)
    warm = iim.Server(opts, budget_bytes=budget, max_slots=slots, ticks_per_run=ticks_per_run, mode=mode,
                      create_threads=create_threads)
    iim.serve(warm, [(0.0, iim.desc_from_spec(sp), sp) for _, sp in trace[:8]], set_data, realtime=False,
              deadline_s=deadline_s, progress=note)
    warm.close()
    S = iim.Server(opts, budget_bytes=budget, max_slots=slots, ticks_per_run=ticks_per_run, mode=mode,
                   create_threads=create_threads)
    arrivals = [(t, iim.desc_from_spec(sp), sp) for t, sp in trace]
    host = {}
    out, wall = iim.serve(S, arrivals, set_data, realtime=True, timings=host, deadline_s=deadline_s, progress=note,
                          data_threads=data_threads)
    stats = S.stats()
    S.close()
    lat = np.array([o[2] for o in out.values()])
    ok = [o for o in out.values() if o[3] == 0 and o[1].converged]
    err = [(o[4].name, o[4].n, o[4].dim, int(o[3]), o[1].iters, o[1].relres) for o in out.values() if o[3] != 0]
    return {
        "solves_per_s": len(ok) / wall, "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()), "wall_s": wall,
        "requests": count, "rate_per_s": rate, "seed": seed, "offered_rate": count / trace[-1][0],
        "completed": len(ok), "failed": len(err), "failures": err[:10], "budget_bytes": budget,
        "peak_bytes": stats["peak_bytes"], "solver": "batched engine" if mode == 0 else
        "per-request solve graphs on streams", "create_threads": create_threads, "client_data_threads": data_threads,
        "problem_reuse": False,
        "host_seconds": {"loop_step": host["step_s"], "client_set_data": host["set_data_s"], "take": host["take_s"],
                         "server_copy_out": stats["host_copy_s"], "server_create_threads": stats["host_create_s"]},
        "requests_2d": sum(1 for _, sp in trace if sp.dim == 2), "requests_3d": sum(1 for _, sp in trace if sp.dim == 3),
    }


def run_serve(args):
    """The serving stream line on its own (2000 requests at 200/s by default)."""
    import torch

    import paper_2503_22455_gb300 as iim
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _load_lib(iim)
    count = args.count or 2000

    def note(t, taken, outstanding, st):
        print(f"serve: {t:.0f} s, {taken} taken, {outstanding} outstanding, states {st['states']}",
              file=sys.stderr, flush=True)

    clocks = Clocks(local)
    clocks.start()
    r = serve_run(iim, torch, count, args.rate, 22455 + rank, slots=args.slots, ticks_per_run=args.ticks_per_run,
                  mode=args.serve_mode, create_threads=args.create_threads, deadline_s=args.serve_deadline, note=note,
                  data_threads=args.data_threads)
    clk = clocks.stop()
    res = {
        "metric": "IIM serving: solves/s and p50/p99 latency (s), rel. resid 1e-10", "value": r["solves_per_s"],
        "unit": "solves/s", "n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "mg_dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serve_poisson_{count}", "rate_per_s": args.rate, "requests": count,
                   "mix": "75% 2D stars n 128..1024, 25% 3D ellipsoids n 64..192; Dirichlet / Neumann; (4,5)/(6,7) 2D",
                   "budget_bytes": r["budget_bytes"], "slots": args.slots, "ticks_per_run": args.ticks_per_run,
                   "tol": 1e-10, "solver": r["solver"]},
        **{k: v for k, v in r.items() if k not in ("solves_per_s",)},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(res))


def ellipsoid_forms(iim, torch, main, flush, n, steps, warmup):
    """The exterior Neumann ellipsoid with a Dirichlet box, (4,5), n^3: per form (FP32
    multigrid, FP32 multigrid with the restricted residuals stored as BF16, all FP64),
    steps of set-up + data + solve to 1e-10, the error against the manufactured solution,
    the device time of one V-cycle and the device bytes the problem holds."""
    import numpy as np

    import workloads as W
    spec = W.ellipsoid_neumann_256(n)
    X = None
    forms = {}
    for name, prec in (("fp32_mg", iim.MG_FP32), ("fp32_mg_bf16_residual", iim.MG_FP32_BF16R),
                       ("fp64", iim.MG_FP64)):
        P = iim.Problem(iim.desc_from_spec(spec), iim.default_options(tol=1e-10, mg_precision=prec), main)
        xc, nc = P.control_points()
        g, _, _ = W.boundary_data(spec, xc.cpu().numpy(), nc.cpu().numpy())
        ph = P.phase().cpu().numpy().astype(bool)
        if X is None:
            X = W.node_coords(n, 3)
            exact = W.to_flat(spec.solution.u_plus(X))
        f = W.to_flat(W.source_term(spec, X, W.from_flat(ph, n, 3)))
        box = W.box_data(spec)
        dv = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        fd, gd, bd = dv(f), dv(g), dv(box)
        x = torch.zeros(P.N, dtype=torch.float64, device="cuda")
        times, iters = [], []
        for k in range(warmup + steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            P.setup()
            P.set_data(fd, gd, None, None, bd)
            x.zero_()
            _, info = P.solve(x)
            b.record(main)
            torch.cuda.synchronize()
            if not info.converged:
                raise RuntimeError(f"{name}: {info.as_dict()}")
            if k >= warmup:
                times.append(a.elapsed_time(b))
                iters.append(info.iters)
        err = float(np.max(np.abs(x.cpu().numpy() - exact)[ph]))
        vc = iim.kernel_time(P, 6, reps=5, flush=flush)
        forms[name] = {"solves_per_s": 1e3 / statistics.mean(times), "ms_per_solve": statistics.mean(times),
                       "iters": statistics.mean(iters), "max_err_vs_exact": err, "vcycle_us": vc,
                       "device_bytes": P.device_bytes()}
        P.close()
        del fd, gd, bd, x
        torch.cuda.empty_cache()
    return {"n": n, "forms": forms, "steps": steps, "warmup": warmup,
            "step": "setup+data+solve of one problem, L2 flushed before each step"}


def circle64_run(iim, torch, main, flush, reps=20, replicas=256):
    """The 64^2 interior Dirichlet circle (4,5), u = exp(x) sin(y): the time of one
    set-up + data + solve alone (latency-bound), and the rate of many replicas of it
    solved together (one solve graph per problem on a pool of streams)."""
    import numpy as np

    import workloads as W
    spec = W.circle_dirichlet_64(64)
    opts = iim.default_options(tol=1e-10)
    P = iim.Problem(iim.desc_from_spec(spec), opts, main)
    f, g, box = _boundary_inputs(P, spec)
    x = torch.zeros(P.N, dtype=torch.float64, device="cuda")
    t, iters = [], []
    for k in range(3 + reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        P.setup()
        P.set_data(f, g, None, None, box)
        x.zero_()
        _, info = P.solve(x)
        b.record(main)
        torch.cuda.synchronize()
        if k >= 3:
            t.append(a.elapsed_time(b))
            iters.append(info.iters)
    ph = P.phase().cpu().numpy().astype(bool)
    ex = W.to_flat(spec.solution.u_plus(W.node_coords(64, 2)))
    err = float(np.max(np.abs(x.cpu().numpy() - ex)[ph]))
    pool = [torch.cuda.Stream() for _ in range(16)]
    probs = [iim.Problem(iim.desc_from_spec(spec), opts, pool[i % 16]) for i in range(replicas)]
    ins = []
    for Q in probs:
        with torch.cuda.stream(Q.stream):
            ins.append(_boundary_inputs(Q, spec))
    xs = [torch.zeros(Q.N, dtype=torch.float64, device="cuda") for Q in probs]
    torch.cuda.synchronize()

    def batch_step():
        start = torch.cuda.Event()
        start.record(main)
        for Q, (fq, gq, bq) in zip(probs, ins):
            Q.stream.wait_event(start)
            with torch.cuda.stream(Q.stream):
                Q.setup()
                Q.set_data(fq, gq, None, None, bq)
        for st in pool:
            main.wait_stream(st)
        infos, _ = iim.batch_solve(probs, xs)
        for st in pool:
            main.wait_stream(st)
        return infos

    batch_step()
    torch.cuda.synchronize()
    bt = []
    for k in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        infos = batch_step()
        b.record(main)
        torch.cuda.synchronize()
        if not all(i.converged for i in infos):
            raise RuntimeError("circle replicas did not converge")
        bt.append(a.elapsed_time(b))
    for Q in probs:
        Q.close()
    P.close()
    return {"us_per_solve": 1e3 * statistics.median(t), "solves_per_s_alone": 1e3 / statistics.median(t),
            "iters": statistics.mean(iters), "max_err_vs_exact": err, "replicas": replicas,
            "replica_solves_per_s": replicas * 1e3 / statistics.mean(bt),
            "step": "setup+data+solve, L2 flushed before each step"}


def run_ellipsoid(args):
    """The 256^3 exterior Neumann ellipsoid line on its own (FP32 / BF16-residual / FP64 forms)."""
    import torch

    import paper_2503_22455_gb300 as iim
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    _load_lib(iim)
    n = args.n if args.n != 1024 else 256
    main = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    r = ellipsoid_forms(iim, torch, main, flush, n, args.steps, args.warmup)
    forms = r["forms"]
    out = {"metric": METRIC, "value": forms["fp32_mg"]["solves_per_s"], "unit": "solves/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms["fp32_mg"]["ms_per_solve"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "mg_dtype": "f32",
           "data": "synthetic",
           "config": {"workload": f"ellipsoid_neumann_{n}_o4", "n": n, "order": 4, "bc": "neumann (exterior)",
                      "box": "dirichlet", "tol": 1e-10, "step": "setup+data+solve"},
           "forms": forms}
    if rank == 0:
        print(json.dumps(out))


def child_line(extra, timeout_s):
    """Run this script with ``extra`` arguments in a child process (its own CUDA context) and
    return the JSON line it prints, or {"error": ...} when it fails or runs past timeout_s
    seconds (the child is killed then)."""
    cmd = [sys.executable, os.path.abspath(__file__), *extra]
    t0 = time.perf_counter()
    try:
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"error": f"killed after {timeout_s} s", "args": extra}
    for line in reversed(p.stdout.splitlines()):
        if line.startswith("{"):
            out = json.loads(line)
            out["child_wall_s"] = time.perf_counter() - t0
            return out
    return {"error": f"exit status {p.returncode}: {p.stderr[-400:]}", "args": extra}


def _load_lib(iim):
    import __graft_entry__ as ge
    try:
        iim.load()
    except ImportError:
        ge.build()
        iim.load()


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2503_22455_gb300 as iim
    _load_lib(iim)
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

    ne = max(1, min(args.engines, B))
    eng_streams = [main] + [torch.cuda.Stream() for _ in range(ne - 1)]
    engines = [iim.Engine(opts, max_slots=B, stream=st) for st in eng_streams] if args.solver == "engine" else None
    engine = engines[0] if engines else None

    def step(s, problems, xvec, use_engine=True):
        """Set-up + data of every problem of the batch on its own stream, then the solves:
        through the batched engine (one graph launch for the whole batch) or one solve
        graph per problem on a stream pool."""
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
        if engines is not None and use_engine:
            # problem i goes to engine i mod ne; the engines run concurrently on their streams
            use = engines[:min(ne, len(problems))]
            t0 = [E.stats()[1] for E in use]
            slots = [use[i % len(use)].admit(P, x) for i, (P, x) in enumerate(zip(problems, xvec))]
            for E in use:
                E.run()
            for E in use:
                E.poll(wait=True)
            infos = [use[i % len(use)].release(sl, x) for i, (sl, x) in enumerate(zip(slots, xvec))]
            for st in eng_streams[1:]:
                main.wait_stream(st)
            kern = iim.launch_count() - l0 - len(use)
            for E, a in zip(use, t0):
                kpt, t1 = E.stats()
                kern += kpt * (t1 - a)
            return infos, kern
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

    def err_of(P, x, s):
        """max error of problem 0's solution at step s against its manufactured solution"""
        spec = inputs[0][2][s]
        ph = P.phase().cpu().numpy().astype(bool)
        Xn = W.node_coords(n, 2)
        ex = W.to_flat(np.where(W.from_flat(ph, n, 2), spec.solution.u_plus(Xn), spec.solution.u_minus(Xn)))
        return float(np.max(np.abs(x.cpu().numpy() - ex)))

    err_exact = err_of(probs[0], xs[0], Wm + K - 1)

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

    forms = {}
    if args.fp64_steps > 0:
        for key, kw in (("fp64_form", {"mg_precision": iim.MG_FP64}),
                        ("w_cycle_form", {"cycle": iim.CYCLE_W}),
                        ("left_gmres_form", {"krylov": iim.KRYLOV_GMRES_LEFT})):
            forms[key] = form_run(args, iim, torch, specs0, streams, step, flush, Wm, main, err_of, kw)
        forms["left_gmres_form"]["tol_on"] = "preconditioned residual |M r| / |M b|"
    other = {}
    if args.other_configs and world == 1:
        other["circle_dirichlet_64_o4"] = circle64_run(iim, torch, main, flush)
        # the larger configurations run in child processes of their own, each with a time
        # limit, so that none of them can hold up this line
        other["ellipsoid_neumann_256_o4"] = child_line(["--workload", "ellipsoid256", "--steps", "2", "--warmup", "1"],
                                                       timeout_s=420)
        other["batch512_mixed_2d"] = child_line(["--workload", "batch512", "--count", "512", "--steps", "2"],
                                                timeout_s=420)
        other["serve_poisson_400"] = child_line(["--workload", "serve", "--count", "400", "--serve-deadline", "240"],
                                                timeout_s=420)
        # the same request mix offered below the loop's capacity: latency when it is not overloaded
        other["serve_poisson_400_rate20"] = child_line(["--workload", "serve", "--count", "400", "--rate", "20",
                                                        "--serve-deadline", "120"], timeout_s=300)
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(probs, torch, inputs, Wm, K, world, main)
    roof = None
    if not args.no_roofline:
        applies = statistics.mean(iters) + 4                  # iterations + start/restarts
        roof = roofline(probs[0], iim, torch, main, applies)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, statistics.mean(iters))
    pk, src = peaks()
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K, "warmup": Wm,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "mg_dtype": "f32", "data": "synthetic",
        "config": workload_config(n, B, f"batched engines x{ne} (lock-step ticks, one graph launch per engine and "
                                        f"step)" if engine is not None else "per-problem solve graphs on a stream pool"),
        "latency_ms_single_solve": statistics.median(lat),
        "iters_mean": statistics.mean(iters), "err_vs_exact": err_exact,
        **forms,
        "other_configs": other or None,
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


def form_run(args, iim, torch, specs0, streams, step, flush, Wm, main, err_of, kw):
    """Another form of the solver (FP64 multigrid, W-cycle or left GMRES), same batch and
    inputs, through per-problem solve graphs (the engine runs the default form only)."""
    import statistics as st
    opts = iim.default_options(tol=1e-10, **kw)
    probs = [iim.Problem(iim.desc_from_spec(sp), opts, s) for sp, s in zip(specs0, streams)]
    xs = [torch.zeros(P.N, dtype=torch.float64, device="cuda") for P in probs]
    step(0, probs, xs, use_engine=False)
    t, it, conv = [], [], True
    for k in range(args.fp64_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        infos, _ = step(Wm + k, probs, xs, use_engine=False)
        b.record(main)
        torch.cuda.synchronize()
        t.append(a.elapsed_time(b))
        it += [inf.iters for inf in infos]
        conv = conv and all(inf.converged for inf in infos)
    err = err_of(probs[0], xs[0], Wm + args.fp64_steps - 1)
    for P in probs:
        P.close()
    return {"value": len(probs) * 1e3 / st.mean(t), "unit": "solves/s", "iters": st.mean(it), "err_vs_exact": err,
            "all_converged": conv}


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


def source_sha(rel_path):
    """First 16 hex digits of the SHA-256 of a source file of the library."""
    import hashlib
    try:
        with open(os.path.join(ROOT, rel_path), "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None


def ncu_traffic():
    """DRAM bytes (read + write) per launch of each profiled kernel, from the ncu captures
    summarised in profiles/: lines "traffic_bytes_per_launch: <kernel> <bytes> <source file>
    <sha16>", the last two naming the file that holds the kernel and its hash when captured.
    A figure whose kernel source has changed since is returned as stale."""
    out = {}
    d = os.path.join(ROOT, "profiles")
    for name in sorted(os.listdir(d)) if os.path.isdir(d) else []:
        try:
            for line in open(os.path.join(d, name)):
                if line.startswith("traffic_bytes_per_launch:"):
                    parts = line.split()
                    fresh = len(parts) >= 5 and source_sha(parts[3]) == parts[4]
                    out[parts[1]] = {"bytes": float(parts[2]), "fresh": fresh, "profile": name}
        except (OSError, ValueError, IndexError):
            continue
    return out


def roofline(P, iim, torch, stream, applies_per_solve):
    """Roofline of the dominant kernel of a solve (by device time per solve), both bound by
    the FP64 pipe: the least-squares fits (once per solve) and the high-order stencil
    (once per operator application).  Timed live with CUDA events on the problem's stream
    over repeated launches of the same kernel on the problem's own data.

    Algorithmic work: fits, per fit of m rows and M monomials, Householder QR
    2 m M^2 - 2/3 M^3 plus w+1 target rows (M^2 for R^-T, 4 m M for Q), summed over the
    launch's fits; stencil, w(2d+1)+1 flop per unknown (16 for the 2D sixth-order
    stencil: pair sums by |j|, then one FMA per |j| and one multiply).
    """
    import ctypes
    lib = iim.load()
    pk, src = peaks()
    peak = fp64_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    out = {}
    us = ctypes.c_double()
    if lib.iim_kernel_time(P.h, 8, 20, ctypes.byref(us)) == 0:
        nfit, rows, M = iim.fit_stats(P)
        w = P.desc.order // 2
        flops = 2.0 * M * M * rows - 2.0 / 3.0 * M ** 3 * nfit + (w + 1) * (M * M * nfit + 4.0 * M * rows)
        out["k_fit_quad"] = {"kernel": f"k_fit_quad<{M}>", "flop": flops, "us": us.value,
                             "us_per_solve": us.value}
    if lib.iim_kernel_time(P.h, 0, 50, ctypes.byref(us)) == 0:
        d, w = P.dim, P.desc.order // 2
        flops = (w * (2 * d + 1) + 1) * P.n_unknowns
        out["k_ho_stencil"] = {"kernel": f"k_ho_stencil<{d},{w}>", "flop": flops, "us": us.value,
                               "us_per_solve": us.value * applies_per_solve}
    if not out:
        return None
    hbm = hbm_kernels(P, iim, torch, pk)
    top = max(out.values(), key=lambda r: r["us_per_solve"])
    achieved = top["flop"] / (top["us"] * 1e-6) / 1e12

    def entry(r):
        a = r["flop"] / (r["us"] * 1e-6) / 1e12
        return {"kernel": r["kernel"], "achieved": a, "frac": a / peak, "us_per_launch": r["us"],
                "flop_per_launch": r["flop"], "us_per_solve": r["us_per_solve"]}

    tr = ncu_traffic().get(top["kernel"])
    traffic = tr["bytes"] if tr and tr["fresh"] else None
    traffic_note = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, profiles/" + tr["profile"]
                    if traffic is not None else
                    "null: no ncu capture of the kernel's current source" if tr is None or not tr["fresh"] else None)
    return {"kernel": top["kernel"], "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s (FP64)",
            "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note, "us_per_launch": top["us"],
            "flop_per_launch": top["flop"],
            "peak_note": "derived FP64 peak: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock (measured 0.598 TFMA/s "
                         "at 1.995 GHz agrees); the measured copy and bf16 peaks do not apply to FP64 work",
            "kernels": [entry(r) for r in out.values()], "hbm_kernels": hbm}


def hbm_kernels(P, iim, torch, pk):
    """Achieved HBM bandwidth of the memory-bound kernels of one iteration: the first level's
    fused multigrid kernels, the stencil and the orthogonalisation passes, each timed alone
    after an L2 flush (inputs from HBM) and back to back (inputs in L2), against the measured
    copy bandwidth.  Algorithmic bytes per node: multigrid down 8 (v) + 1 (class: unknown,
    irregular, phase) + 4 (f) + 4 (u) + 1 (coarse f); up 4 (u) + 4 (f) + 1 (class) +
    1 (coarse u) + 8 (z); stencil 8 (u) + 8 (w) + 1 (phase); multi-dot and update over
    j + 1 = restart/2 + 1 vectors: 8 (j + 2) and 8 (j + 3)."""
    peak = pk.get("hbm_gbs")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    N, j = P.N, P.options.restart // 2
    rb = "16,4" if P.n >= 2048 else ("16,2" if P.n >= 512 else "8,2")
    cases = [("mg_down0", f"k_mg2d_rb<float,{rb},0> first level (down)", 18),
             ("mg_up0", f"k_mg2d_rb<float,{rb},1> first level (up)", 18),
             ("stencil", "k_ho_stencil", 17),
             ("multidot", f"k_multidot<{j + 1}>", 8 * (j + 2)),
             ("update", f"k_update<{j + 1}>", 8 * (j + 3))]
    res = []
    for which, name, bpn in cases:
        try:
            cold = iim.kernel_time(P, which, reps=10, flush=flush)
            warm = iim.kernel_time(P, which, reps=50)
        except iim.IIMError:
            continue
        b = bpn * N
        r = {"kernel": name, "bytes_per_launch": b, "us_hbm": cold, "gbs_hbm": b / cold / 1e3,
             "us_l2": warm, "gbs_l2": b / warm / 1e3}
        if peak:
            r["frac_hbm"] = r["gbs_hbm"] / peak
        res.append(r)
    try:
        res.append({"kernel": "k_vcycle_tail (one CTA, latency)", "us_l2": iim.kernel_time(P, "mg_tail", reps=50)})
    except iim.IIMError:
        pass
    del flush
    return res


# ------------------------------------------------------------------------------ the CPU oracle
def _oracle_worker(task):
    """One oracle problem in a worker process: set-up (operator, data, multigrid, right-hand
    side) and FGMRES(10) to tol 1e-10 or max_iter iterations.  Returns the set-up and
    FGMRES times, the iterations run, and the mean time of one operator application and of
    one preconditioner application inside FGMRES."""
    n, seed, max_iter = task
    import workloads as W
    from oracle.fgmres import fgmres
    from oracle.problem import OracleProblem
    t0 = time.perf_counter()
    O = OracleProblem(W.star_interface_variant(n, seed))
    f, data = O.data()
    _ = O.mg
    b = O.op.rhs(f, data)
    t1 = time.perf_counter()
    acc = {"A": [0.0, 0], "M": [0.0, 0]}

    def timed(key, fn):
        def g(v):
            a = time.perf_counter()
            out = fn(v)
            acc[key][0] += time.perf_counter() - a
            acc[key][1] += 1
            return out
        return g
    _, info = fgmres(timed("A", O.op.apply), timed("M", O.precondition), b, tol=1e-10, restart=10,
                     max_iter=max_iter)
    t2 = time.perf_counter()
    return {"setup": t1 - t0, "fgmres": t2 - t1, "iters": int(info["iters"]),
            "t_apply": acc["A"][0] / max(acc["A"][1], 1), "t_precond": acc["M"][0] / max(acc["M"][1], 1)}


def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"


class OraclePool:
    """The oracle on the host's cores: one worker process per core (spawned, so that it is
    independent of any CUDA state of the parent), each solving its own problem."""

    def __init__(self, n, cores=None):
        import multiprocessing as mp
        self.n = n
        self.cores = cores or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_worker_init)

    def run(self, seeds, max_iter):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(self.n, s, max_iter) for s in seeds], chunksize=1)
        return time.perf_counter() - t0, res

    def close(self):
        self.pool.terminate()
        self.pool.join()


def cpu_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "lscpu_model": model}


def solve_fraction(r, iters_full, restart=10):
    """The part of one complete solve a sample r did: its measured time over the time of a
    complete solve, modelled from the sample's own set-up time and its mean operator and
    preconditioner times (per iteration one of each, plus one operator application at the
    start and after each restart cycle)."""
    cycles = -(-iters_full // restart)
    full = r["setup"] + iters_full * (r["t_apply"] + r["t_precond"]) + (1 + cycles) * r["t_apply"]
    return (r["setup"] + r["fgmres"]) / full


def oracle_step(pool, seeds, iters_full, sample_iters=2):
    """One step on every worker: its own problem's set-up and sample_iters iterations.
    Returns (wall seconds, solves done = sum of the solve fractions)."""
    wall, res = pool.run(seeds, sample_iters)
    return wall, sum(solve_fraction(r, iters_full) for r in res)


def cpu_baseline(n, gpu_iters):
    """The oracle on the host, a bounded sample of the headline workload: on all cores
    (one problem per core) and on one core, each sample a set-up plus two FGMRES
    iterations, scaled by its measured set-up, operator and preconditioner times to a
    solve of the GPU's iteration count."""
    full = max(1, round(gpu_iters))
    allc = OraclePool(n)
    try:
        allc.run(list(range(allc.cores)), 1)                       # imports, first touch
        wall, done = oracle_step(allc, [100 + i for i in range(allc.cores)], full)
    finally:
        allc.close()
    one = OraclePool(n, cores=1)
    try:
        w1, d1 = oracle_step(one, [100], full)
    finally:
        one.close()
    return {"value": done / wall, "unit": "solves/s", "cores": allc.cores, "kind": "oracle",
            "sample": f"one {n}^2 problem per core ({allc.cores} worker processes): oracle set-up + 2 FGMRES "
                      f"iterations each ({wall:.1f} s wall), scaled by the measured set-up, operator and "
                      f"preconditioner times to solves of {full} iterations",
            "one_thread": {"value": d1 / w1, "unit": "solves/s", "cores": 1, "seconds": w1},
            **cpu_info()}


def run_reference(args):
    """The CPU oracle on the headline workload (the reference arm).  First warm-up step:
    one complete solve to 1e-10 per core (the oracle's own iteration count and a measured
    complete-solve rate).  Every other step: on each core, its own problem's set-up and two
    FGMRES iterations, counted as the part of a complete solve it is (measured times)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    pool = OraclePool(args.n)
    try:
        seeds = lambda k: [1000 * k + i for i in range(pool.cores)]
        wall_full, res = pool.run(seeds(0), 100000)
        iters_full = max(r["iters"] for r in res)
        complete = {"value": len(res) / wall_full, "unit": "solves/s", "seconds": wall_full,
                    "iters": [r["iters"] for r in res],
                    "model_vs_measured": [round(solve_fraction(r, r["iters"]), 3) for r in res]}
        for k in range(1, args.warmup):
            oracle_step(pool, seeds(k), iters_full)
        walls, done = [], 0.0
        for k in range(args.steps):
            w, d = oracle_step(pool, seeds(args.warmup + k), iters_full)
            walls.append(w)
            done += d
    finally:
        pool.close()
    value = done / sum(walls)
    cfg = workload_config(args.n, args.batch, "CPU oracle: numpy/scipy FP64, one problem per core")
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": cfg,
           "cpu_baseline": {"value": value, "unit": "solves/s", "kind": "oracle", "cores": pool.cores,
                            "sample": f"per step: one {args.n}^2 problem per core, set-up + 2 FGMRES iterations, "
                                      f"scaled by the measured set-up, operator and preconditioner times to "
                                      f"solves of {iters_full} iterations"},
           "complete_solves": complete, **cpu_info(),
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batch512":
        run_batch(a)
    elif a.workload == "serve":
        run_serve(a)
    elif a.workload == "ellipsoid256":
        run_ellipsoid(a)
    else:
        run_ours(a)
