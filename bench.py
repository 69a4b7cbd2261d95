#!/usr/bin/env python
"""Benchmark of the parareal + splitting solver on one node.

One step = one complete solve of the workload to tolerance through the C ABI:
the sequential coarse sweep, every parareal iteration (batched fine propagator
over all slices, coarse chain with the fused correction, increment test) until
the stopping rule fires.  Inputs are resident in HBM before the timed region.

value    unknown-updates/s over the K timed solves (all ranks): interior unknowns
         advanced by one step (FIE; DR for the fine steps with --fine dr), summed over the
         fine and coarse work executed.
e2e      the same through ps_run_parareal_host with the initial state in pinned host
         memory and U_N copied back every step.
roofline the dominant kernel's algorithmic bytes (or flops) per launch over its
         average CUDA-event duration in the timed region, against the measured peak.

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
Multi-GPU (torchrun): every rank solves its own copy (replicas, weak scaling); only the
timing uses collectives.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unknown-updates/s & HBM roofline % of split sweeps; time-to-tol vs plain FP64 GPU"
UNIT = "unknown-updates/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 FMA issue rate of this GB300 pool, measured with a dependent-free DFMA loop
# (152 SMs x 256 threads x 8 chains): 0.595e12 FMA/s = 1.19 TFLOP/s (FMA = 2 flops).
FP64_PEAK_TFLOPS = 1.19


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per node-slice of the fine tile
# sweeps, from one ncu capture of the kernel built from the kernel source with this hash prefix
# (127^3 x 64 slices, scaled to any launch by the node-slices it processes).  A kernel whose
# source changed since is reported with traffic null.
_UNITS_127 = 127 ** 3 * 64
TRAFFIC = {"F.x.f32": {"bytes_per_node_slice": (549.214464e6 + 463.244544e6) / _UNITS_127, "tile_src_sha": "b27d5c80c1ebe8be"},
           "F.y.f32": {"bytes_per_node_slice": (541.012224e6 + 463.005696e6) / _UNITS_127, "tile_src_sha": "b27d5c80c1ebe8be"},
           "F.z.f32": {"bytes_per_node_slice": (541.032448e6 + 462.982912e6) / _UNITS_127, "tile_src_sha": "b27d5c80c1ebe8be"}}


def tile_src_sha():
    """Hash of the single-problem tile kernel's source: the async-copy helpers and ps_tile.cu up to
    the persistent and grouped variants (the line solve, the tile body, tile_sweep_kernel)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2502_08370_gb300", "csrc")
    with open(os.path.join(csrc, "ps_async.h")) as f:
        helpers = f.read()
    with open(os.path.join(csrc, "ps_tile.cu")) as f:
        tile = f.read()
    return hashlib.sha256((helpers + tile[:tile.index("// Persistent form")]).encode()).hexdigest()[:16]


def workload(name):
    from paper_2502_08370_gb300 import workloads as wl
    if name == "heat3d_255":
        return wl.heat3d_255()
    if name == "heat2d_63":
        return wl.heat2d_63()
    if name == "dd2d_1023":
        # run to its tolerance 1e-10 (or to k = N, where parareal is the sequential fine solution)
        return wl.dd2d_1023()
    if name.startswith("dd_scal99_q"):
        # the scalability experiment of Sec. 5.1: 99^2, DeltaT = 1/32, delta t = 1/3200, F with q = 2
        # strips (overlap 1/16), G with q strips (overlap 1/32), five iterations from u = 0
        q = int(name[len("dd_scal99_q"):])
        n, T, N, s = 99, 1.0, 32, 100
        S, st, exact = wl.manufactured((n, n), T, N, s)
        return dict(n=(n, n), a=None, c=0.0, src=S, src_t=st, u0=np.zeros((n, n)), T=T, N=N, g=1, s=s, tol=0.0,
                    max_iter=5, split="dd", boxes=(4, 1), overlap=1 / 16, coarse_boxes=(2 * q, 1),
                    coarse_overlap=1 / 32, exact=exact)
    if name == "adjoint2d_511":
        return wl.adjoint2d_511()
    if name == "batch256":
        return {"batch": wl.batch256(), "n": (0, 0), "split": "dim", "N": 0, "g": 1, "s": 0, "T": 1.0,
                "tol": 1e-8}
    if name.startswith("heat3d_"):
        return wl.heat3d_255(n=int(name.split("_")[1]))
    raise SystemExit(f"unknown workload {name}")


def dist_setup(backend):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return rank, ws


def combine_ranks(ms, units, device):
    """Whole-job figures of a replicas run: the slowest rank's time and the units of all ranks
    (one rank: unchanged).  device: where the collective's tensor lives ("cuda" for NCCL,
    "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms), float(units)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


TILE_KW = {}  # fine tile shape overrides from the command line (tile_positions, tile_slots, ...)
PROB_KW = {}  # other problem options from the command line (overlap_phases)
AUTOTUNE = {"on": True, "seconds": 0.0}  # run ps_autotune on each single problem before timing it


def make_problem(ps, torch, cfg, precision, timing, coarse_mode="fp64", fine_method="fie", tune=True):
    grid = ps.Grid(cfg["n"])
    a = None if cfg["a"] is None else torch.as_tensor(cfg["a"]).cuda()
    src = None if cfg["src"] is None else torch.as_tensor(cfg["src"]).cuda()
    op = ps.Operator(grid, a=a, c=cfg["c"], src=src, src_t=cfg["src_t"])
    sp = ps.Splitting(op, cfg["split"], cfg.get("boxes", (1, 1)), cfg.get("overlap", 0.0))
    spc = ps.Splitting(op, cfg["split"], cfg["coarse_boxes"], cfg["coarse_overlap"]) if "coarse_boxes" in cfg \
        else None
    prob = ps.Problem(sp, cfg["T"], cfg["N"], cfg["g"], cfg["s"], coarse=spc, precision=precision, timing=timing,
                      coarse_mode=coarse_mode, fine_method=fine_method, **TILE_KW, **PROB_KW)
    prob._keep = (grid, op, sp, spc, a, src)
    if tune and AUTOTUNE["on"] and not any(v not in (0, "auto") for v in TILE_KW.values()):
        t0 = time.perf_counter()
        prob.autotune(budget_ms=150)
        AUTOTUNE["seconds"] += time.perf_counter() - t0
        prob._tuned = prob.autotune_record()
    return prob


def time_fie_fie_to_tol(ps, torch, cfg, u0, stream, reps=2):
    """Parareal/FIE-FIE in FP64 on the workload: mean device time of `reps` solves to the
    workload's tolerance after one untimed solve; returns (ms, iterations, U_N on the host)."""
    q = make_problem(ps, torch, cfg, "fp64", timing=0, fine_method="fie")
    q.run(u0, cfg["tol"])
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(reps):
        it = q.run(u0, cfg["tol"])
    c1.record(stream)
    torch.cuda.synchronize()
    uN = q.state(cfg["N"]).cpu().numpy()
    return c0.elapsed_time(c1) / reps, it, uN


def fine_steps_fn(fine):
    import oracle as orc
    return (orc.propagate_dr, "DR") if fine == "dr" else (orc.propagate, "FIE")


def cpu_sample(cfg, seconds, fine="fie"):
    """The oracle, as it stands, on a bounded sample: whole fine steps (FIE, or DR for
    Parareal/FIE-DR) of one slice."""
    import numpy as np

    import oracle as orc
    orp = orc.Problem(cfg["n"], a=cfg["a"], c=cfg["c"], src=cfg["src"], src_t=cfg["src_t"], split=cfg["split"],
                      boxes=cfg.get("boxes", (1, 1)), overlap=cfg.get("overlap", 0.0))
    tau = cfg["T"] / cfg["N"] / cfg["s"]
    u = np.ascontiguousarray(cfg["u0"], dtype=np.float64)
    t = time.perf_counter()
    step_fn, kind = fine_steps_fn(fine)
    u = step_fn(orp, tau, 1, u, t0=0)
    one = time.perf_counter() - t
    steps = max(1, int(seconds / max(one, 1e-6)))
    t = time.perf_counter()
    step_fn(orp, tau, steps, u, t0=1)
    dt = time.perf_counter() - t
    nt = int(np.prod(cfg["n"]))
    grid = "x".join(str(v) for v in cfg["n"])
    return {"value": steps * nt / dt, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
            "sample": f"{steps} fine {kind} steps of one {grid} slice ({len(cfg['n'])} line-solve substeps each), "
                      f"{dt:.1f} s"}


def run_reference(args, cfg, rank, ws):
    """The oracle as it stands: each step is one fine step (FIE, or DR with --fine dr) of one
    slice of the workload."""
    if rank != 0:
        return
    import numpy as np

    import oracle as orc
    orc.build()
    orp = orc.Problem(cfg["n"], a=cfg["a"], c=cfg["c"], src=cfg["src"], src_t=cfg["src_t"], split=cfg["split"],
                      boxes=cfg.get("boxes", (1, 1)), overlap=cfg.get("overlap", 0.0))
    tau = cfg["T"] / cfg["N"] / cfg["s"]
    u = np.ascontiguousarray(cfg["u0"], dtype=np.float64)
    step_fn, kind = fine_steps_fn(getattr(args, "fine", "fie"))
    for w in range(args.warmup):
        u = step_fn(orp, tau, 1, u, t0=w)
    t = time.perf_counter()
    for k in range(args.steps):
        u = step_fn(orp, tau, 1, u, t0=args.warmup + k)
    dt = time.perf_counter() - t
    nt = int(np.prod(cfg["n"]))
    value = args.steps * nt / dt
    grid = "x".join(str(v) for v in cfg["n"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, cfg),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                             "sample": f"each step: one fine {kind} step ({len(cfg['n'])} line-solve substeps) of one "
                                       f"{grid} slice of the workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, cfg):
    if "batch" in cfg:
        b = cfg["batch"]
        tot = sum(int(np.prod(c["n"])) * (2 * c["N"] + 1) * 8 for c in b)
        return {"workload": args.workload, "problems": len(b), "grids": "nx, ny from {63,127,255,511}",
                "N_slices": "{8,16,32,64}", "fine_steps": "16..128", "tol": cfg["tol"], "precision": "mixed",
                "coarse": getattr(args, "coarse", "fp64"),
                "l2": f"inputs larger than L2 ({tot / 1e9:.1f} GB of slice states)"}
    grid = "x".join(str(v) for v in cfg["n"])
    nt = int(np.prod(cfg["n"]))
    gb = nt * (3 * cfg["N"] + 1) * 8 / 1e9
    out = {"workload": args.workload, "grid": grid, "splitting": cfg["split"], "N_slices": cfg["N"],
           "coarse_steps": cfg["g"], "fine_steps": cfg["s"], "T": cfg["T"], "tol": cfg["tol"],
           "precision": args.precision, "coarse": getattr(args, "coarse", "fp64"),
           "fine": "dr" if getattr(args, "fine", "fie") == "dr" else "fie",
           "tiles": {k: v for k, v in TILE_KW.items() if v not in (0, "auto")} or "auto",
           **({"overlap_phases": True} if PROB_KW.get("overlap_phases") else {}),
           "l2": (f"inputs larger than L2 ({gb:.1f} GB of slice states streamed per step)" if gb > 0.2 else
                  f"working set {gb * 1e3:.0f} MB fits in L2: latency-bound case, no roofline claim")}
    if cfg["split"] == "dd":
        out["boxes"] = list(cfg["boxes"])
        out["overlap"] = cfg["overlap"]
        if "coarse_boxes" in cfg:
            out["coarse_boxes"] = list(cfg["coarse_boxes"])
            out["coarse_overlap"] = cfg["coarse_overlap"]
    if cfg.get("max_iter"):
        out["max_iter"] = cfg["max_iter"]
    return out


def finish_line(args, cfg, value, ms_per_step, launches, extra, rank, ws, e2e=None, roof=None, cpu=None,
                dtype="f64", clocks=None):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic", "config": config_of(args, cfg), "clocks": clocks, "e2e": e2e,
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, cfg, ps, torch, rank, ws):
    """256 independent problems: batched (grouped launches + graph) vs one at a time."""
    cfgs = cfg["batch"]
    # the batch's own autotuner (after creation) keeps each problem on the batch's schedules
    probs = [make_problem(ps, torch, c, "mixed", timing=0, coarse_mode=args.coarse, tune=False) for c in cfgs]
    u0s = [torch.as_tensor(c["u0"]).cuda() for c in cfgs]
    batch = ps.Batch(probs)
    t0 = time.perf_counter()
    chosen = batch.autotune(budget_ms=15)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.run(u0s, cfg["tol"])
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) if rank == 0 else None
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    upd, launches, its = 0.0, 0, None
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        its = batch.run(u0s, cfg["tol"])
        st = batch.stats()
        upd += st["unknown_updates"]
        launches += st["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    # one problem after another through ps_run_parareal (same results, bitwise)
    torch.cuda.synchronize()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for p, u in zip(probs, u0s):
        p.run(u, cfg["tol"])
    c1.record(stream)
    torch.cuda.synchronize()
    seq_ms = c0.elapsed_time(c1)
    # end to end: initial states from pinned host memory, every U_N back to the host
    hosts = [torch.as_tensor(c["u0"]).contiguous().pin_memory() for c in cfgs]
    outs = [torch.empty_like(h).pin_memory() for h in hosts]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    e2e_upd = 0.0
    for _ in range(args.steps):
        devs = [h.cuda(non_blocking=True) for h in hosts]
        batch.run(devs, cfg["tol"])
        e2e_upd += batch.stats()["unknown_updates"]
        for p, o in zip(probs, outs):
            o.copy_(p.state(p.N), non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1)
    nbytes = sum(int(np.prod(c["n"])) * 8 for c in cfgs)
    e2e = {"value": e2e_upd / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
           "wall_s": time.perf_counter() - w0}
    extra = {"time_to_tol": {"batched_ms": ms / args.steps, "one_at_a_time_ms": seq_ms,
                             "speedup_vs_one_at_a_time": seq_ms / (ms / args.steps),
                             "iterations_min_max": [min(its), max(its)]},
             "autotune": {"seconds": tune_s, "classes": len(chosen),
                          "choices": sorted({v for v in chosen.values()})},
             "roofline_note": "the batch replays graphs of grouped launches; per-kernel rooflines are those of "
                              "the single-problem workloads"}
    finish_line(args, cfg, upd / (ms / 1e3), ms / args.steps, launches, extra, rank, ws, e2e=e2e, dtype="f32+f64",
                clocks=clocks)


def run_adjoint(args, cfg, ps, torch, rank, ws):
    """Gradient of J = 1/2 ||U_N - target||^2 w.r.t. u0 and the nodal coefficient a."""
    n = cfg["n"]
    nt = int(np.prod(n))
    grid = ps.Grid(n)
    a = torch.as_tensor(cfg["a"]).cuda()
    op = ps.Operator(grid, a=a)
    sp = ps.Splitting(op)
    prob = ps.Problem(sp, cfg["T"], cfg["N"], 1, cfg["s"], tol_mode=1, timing=1)
    u0 = torch.as_tensor(cfg["u0"]).cuda()
    tol = cfg["tol"]
    prob.update_coefficients(torch.as_tensor(cfg["a_target"]).cuda())
    prob.run(u0, tol)
    tgt = prob.state(cfg["N"]).clone()
    prob.update_coefficients(a)
    stream = torch.cuda.current_stream()

    M = len(n)

    def gradient():
        prob.run(u0, tol)
        fwd = prob.stats()
        gN = prob.state(cfg["N"]) - tgt
        gu, ga = prob.vjp(gN, tol)
        adj = prob.stats()  # the adjoint parareal's own counts
        # + recomputation and backward sweeps of every slice: 2 packs, s*M sweeps, s*M transposed
        # sweeps and s*M edge-product kernels, one combine
        nl = fwd["kernel_launches"] + adj["kernel_launches"] + 3 + 3 * cfg["s"] * M
        return gu, ga, fwd["unknown_updates"] + adj["unknown_updates"] + 2.0 * cfg["N"] * cfg["s"] * nt, nl

    for _ in range(args.warmup):
        gradient()
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) if rank == 0 else None
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    upd, launches = 0.0, 0
    e0.record(stream)
    for _ in range(args.steps):
        gu, ga, u, nl = gradient()
        upd += u
        launches += nl
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    # Central differences of J on seeded unit directions: the fourth-order stencil
    #   D(e) = [8 (J(+e) - J(-e)) - (J(+2e) - J(-2e))] / (12 e)
    # at e and e/2, combined as (16 D(e/2) - D(e)) / 15 (sixth order),
    # of the discrete forward map the adjoint differentiates (N*s fine steps from u0).  U_N carries
    # ~1e-15 relative rounding after 2048 steps; divided by e and concentrated by the cancellation
    # in J, that noise is ~1e-5 of the derivative at e = 1e-4 and ~1e-7 at e = 0.1, where each node
    # moves by e / sqrt(#nodes) ~ 2e-4 and the stencil's truncation stays near 1e-8.
    from paper_2502_08370_gb300 import workloads as wl

    # the gradient the finite differences check is the exact one of the forward map: forward and
    # adjoint parareal run to k = N (finite termination, Sec. 3); the timed gradient at the
    # workload's tolerance is compared with it
    prob.run(u0, tol)
    gu_tol, ga_tol = prob.vjp(prob.state(cfg["N"]) - tgt, tol)
    prob.run(u0, 0.0)
    gN = prob.state(cfg["N"]) - tgt
    gu, ga = prob.vjp(gN, 0.0)
    tol_gap = {"a": float((ga_tol - ga).abs().max() / ga.abs().max()),
               "u0": float((gu_tol - gu).abs().max() / gu.abs().max())}
    nsteps = cfg["N"] * cfg["s"]

    def J_of(aa, uu):
        prob.update_coefficients(aa)
        x = uu.clone()
        prob.propagate(0, nsteps, x)
        r = x - tgt
        return 0.5 * float((r * r).sum())

    def fd6(f, eps):
        # fourth-order central differences at eps and eps/2 combined to sixth order (Richardson)
        memo = {}

        def F(e):
            if e not in memo:
                memo[e] = f(e)
            return memo[e]

        def fd4(h):
            return (8.0 * (F(h) - F(-h)) - (F(2 * h) - F(-2 * h))) / (12.0 * h)

        return (16.0 * fd4(eps / 2) - fd4(eps)) / 15.0

    errs_a, errs_u = [], []
    eps = 0.4
    for d in wl.random_directions(tuple(a.shape), args.fd_dirs, cfg["dirs_seed"]):
        dd = torch.as_tensor(d).cuda()
        fd = fd6(lambda e: J_of(a + e * dd, u0), eps)
        errs_a.append(abs(float((ga * dd).sum()) - fd) / abs(fd))
    for d in wl.random_directions(tuple(u0.shape), 5, cfg["dirs_seed"] + 1):
        dd = torch.as_tensor(d).cuda()
        fd = fd6(lambda e: J_of(a, u0 + e * dd), eps)
        errs_u.append(abs(float((gu * dd).sum()) - fd) / abs(fd))
    prob.update_coefficients(a)
    extra = {"gradient": {"ms_per_gradient": ms / args.steps, "fd_directions_a": len(errs_a),
                          "fd_stencil": "4-point central at eps and eps/2, Richardson-extrapolated (6th order)", "fd_eps": eps,
                          "fd_max_rel_err_a": max(errs_a), "fd_median_rel_err_a": float(np.median(errs_a)),
                          "fd_dirs_within_1e-6_a": int(sum(e <= 1e-6 for e in errs_a)),
                          "fd_rel_errs_a": errs_a,
                          "fd_directions_u0": len(errs_u),
                          "fd_max_rel_err_u0": max(errs_u),
                          "fd_gradient": "exact (forward and adjoint parareal to k = N)",
                          "rel_maxnorm_gap_gradient_at_tol_vs_exact": tol_gap,
                          "adjoint_parareal_iters": getattr(prob, "last_adjoint_iters", None)}}
    finish_line(args, cfg, upd / (ms / 1e3), ms / args.steps, launches, extra, rank, ws, clocks=clocks)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="heat3d_255")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--coarse", default="fp64", choices=["delta32", "fp64"],
                    help="coarse propagator of the mixed form: FP64 (default: the parareal defect, correction and "
                         "test all in FP64), or the FP32 increment form (dimensional splitting)")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain FP64 time-to-tolerance run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--fd-dirs", type=int, default=20, help="finite-difference directions (adjoint workload)")
    ap.add_argument("--fine", default="fie", choices=["fie", "dr"],
                    help="fine propagator: FIE steps, or Douglas-Rachford steps (Parareal/FIE-DR, FP64, "
                         "dimensional or DD splitting)")
    ap.add_argument("--slices", type=int, default=0,
                    help="override the workload's slice count N (small-footprint profiling runs; named in config)")
    ap.add_argument("--tile-positions", type=int, default=0, help="fine tiles: line positions per tile (0 = auto)")
    ap.add_argument("--tile-slots", type=int, default=0, help="fine tiles: time slices per tile (0 = auto)")
    ap.add_argument("--tile-lines-per-thread", type=int, default=0, help="fine FP32 tiles: lines per thread (0 = auto)")
    ap.add_argument("--coarse-sweep", default="auto", choices=["auto", "staged", "streamed"],
                    help="coarse line solves on one slice: staged through shared memory or streamed")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedules (no ps_autotune)")
    ap.add_argument("--overlap-phases", action="store_true",
                    help="run the fine phase slot group by slot group beside the coarse chain (same values)")
    args = ap.parse_args()
    AUTOTUNE["on"] = not args.no_autotune
    if args.overlap_phases:
        PROB_KW["overlap_phases"] = True
    TILE_KW.update(tile_positions=args.tile_positions, tile_slots=args.tile_slots,
                   tile_lines_per_thread=args.tile_lines_per_thread, coarse_sweep=args.coarse_sweep)
    if args.warmup < 3:
        args.warmup = 3
    cfg = workload(args.workload)
    if args.slices > 0 and "batch" not in cfg:
        cfg["N"] = args.slices

    if args.workload in ("heat2d_63", "dd2d_1023", "adjoint2d_511") or args.workload.startswith("dd_scal99"):
        args.precision = "fp64"  # these workloads are specified in FP64
        args.no_compare = True
    if args.fine == "dr":
        if "batch" in cfg or args.workload == "adjoint2d_511":
            raise SystemExit("--fine dr runs the single-problem workloads (dimensional or DD splitting)")
        args.precision = "fp64"  # the DR fine propagator runs in FP64
        args.no_compare = True
    if args.precision == "fp64" or cfg.get("split") == "dd":
        args.coarse = "fp64"

    if args.impl == "reference":
        rank, ws = dist_setup("gloo")
        run_reference(args, cfg, rank, ws)
        return

    import numpy as np
    import torch

    import paper_2502_08370_gb300 as ps
    from paper_2502_08370_gb300 import build as psbuild
    rank, ws = dist_setup("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        psbuild.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    ps.lib()
    if args.workload == "batch256":
        return run_batch(args, cfg, ps, torch, rank, ws)
    if args.workload == "adjoint2d_511":
        return run_adjoint(args, cfg, ps, torch, rank, ws)

    prob = make_problem(ps, torch, cfg, args.precision, timing=2, coarse_mode=args.coarse, fine_method=args.fine)
    tuned = getattr(prob, "_tuned", [])
    max_iter = cfg.get("max_iter", 0)
    u0 = torch.as_tensor(cfg["u0"]).cuda()
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        prob.run(u0, cfg["tol"], max_iter)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(local) if rank == 0 else None
    updates = 0.0
    launches = 0
    iters = []
    kern = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        iters.append(prob.run(u0, cfg["tol"], max_iter))
        st = prob.stats()
        updates += st["unknown_updates"]
        launches += st["kernel_launches"]
        for name, k in prob.kernel_times().items():
            acc = kern.setdefault(name, dict(launches=0, ms=0.0, bytes=0.0, flops=0.0))
            for key in acc:
                acc[key] += k[key]
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    ms_max, updates_all = combine_ranks(ms, updates, "cuda")
    value = updates_all / (ms_max / 1000.0)
    uN_mixed = prob.state(cfg["N"]).cpu().numpy()

    # dominant kernel and its roofline
    pk, pk_kind = load_peaks()
    dom_name, dom = max(kern.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = dom["ms"] / dom["launches"]
    # FP64 sweeps and the DR stencil are bound by the FP64 issue rate; the DR add pass by HBM
    is_f64 = (dom_name.endswith("f64") or "f64+" in dom_name) and not dom_name.startswith("F.dradd")
    if is_f64:
        achieved = dom["flops"] / dom["launches"] / (per_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None}
    else:
        achieved = dom["bytes"] / dom["launches"] / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None}
        tr = TRAFFIC.get(dom_name)
        if tr and tr["tile_src_sha"] == tile_src_sha():
            # fine sweep bytes = node-slices x (4 in + 4 out) + the line factors l, r (FP32, per node)
            # (+ the source row, 8 B per node, on the x sweep that adds it)
            nt = float(np.prod(cfg["n"]))
            src_b = 8.0 * nt if (dom_name.startswith("F.x") and cfg.get("src") is not None) else 0.0
            node_slices = (dom["bytes"] / dom["launches"] - 8.0 * nt - src_b) / 8.0
            roof["traffic"] = tr["bytes_per_node_slice"] * node_slices
    roof.update({"kernel": dom_name, "launches_timed": dom["launches"], "ms_per_launch": per_launch_ms,
                 "algorithmic_bytes_per_launch": dom["bytes"] / dom["launches"],
                 "share_of_step": dom["ms"] / ms, "peak_source": pk_kind})
    kernels = {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                   "GB/s": round(v["bytes"] / max(v["ms"], 1e-9) / 1e6, 1),
                   "TFLOP/s": round(v["flops"] / max(v["ms"], 1e-9) / 1e9, 4)}
               for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms"])}

    # end to end through the host entry point (pinned host buffers)
    nt = int(np.prod(cfg["n"]))
    u0h = torch.as_tensor(cfg["u0"]).contiguous().pin_memory()
    uNh = torch.empty_like(u0h).pin_memory()
    prob_e2e = prob
    prob_e2e.run_host(u0h, uNh, cfg["tol"], max_iter)
    torch.cuda.synchronize()
    barrier()
    e2e_upd = 0.0
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        prob_e2e.run_host(u0h, uNh, cfg["tol"], max_iter)
        e2e_upd += prob_e2e.stats()["unknown_updates"]
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_wall = time.perf_counter() - t0
    barrier()
    e2e_ms, e2e_upd = combine_ranks(e2e_ms, e2e_upd, "cuda")
    e2e = {"value": e2e_upd / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": 8 * nt,
           "d2h_bytes_per_step": 8 * nt, "wall_s": e2e_wall}

    # plain FP64 GPU method: time to tolerance at the same tolerance; the other FP32 form; and the
    # accuracy of every arm against one common reference
    compare = None
    accuracy = None
    if not args.no_compare and args.precision != "fp64":
        del prob
        torch.cuda.empty_cache()

        def time_to_tol(precision, coarse_mode, s_fine=None, reps=2, timing=2):
            c = dict(cfg) if s_fine is None else dict(cfg, s=s_fine)
            q = make_problem(ps, torch, c, precision, timing=timing, coarse_mode=coarse_mode)
            q.run(u0, c["tol"])
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(reps):
                it = q.run(u0, c["tol"])
            c1.record(stream)
            torch.cuda.synchronize()
            t = c0.elapsed_time(c1) / reps
            out = {"ms": t, "iters": it, "uN": q.state(c["N"]).cpu().numpy(),
                   "ups": q.stats()["unknown_updates"] / (t / 1000.0), "kern": q.kernel_times() if timing >= 2 else {}}
            del q
            torch.cuda.empty_cache()
            return out

        def rel(a, b):
            return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

        plain = time_to_tol("fp64", "fp64")
        # the FP64 comparator against GB300's FP64 issue rate: its dominant kernel and the whole solve
        pk_name, pk = max(plain["kern"].items(), key=lambda kv: kv[1]["ms"])
        tot_flops = sum(k["flops"] for k in plain["kern"].values())
        tot_ms = sum(k["ms"] for k in plain["kern"].values())
        fp64_pipe = {"kernel": pk_name, "TFLOP/s": pk["flops"] / pk["ms"] / 1e9,
                     "frac": pk["flops"] / pk["ms"] / 1e9 / FP64_PEAK_TFLOPS,
                     "solve_TFLOP/s": tot_flops / tot_ms / 1e9, "solve_frac": tot_flops / tot_ms / 1e9 / FP64_PEAK_TFLOPS,
                     "peak_TFLOP/s": FP64_PEAK_TFLOPS, "peak_source": "measured DFMA rate of this GPU pool"}
        forms = {"fp64": "FP32 fine line solves; FP64 coarse propagator, parareal defect, correction and test",
                 "delta32": "FP32 fine line solves; coarse increment form: FP32 line solves on the FP32-rounded "
                            "increment, FP64 correction and test"}
        other_mode = "delta32" if args.coarse == "fp64" else "fp64"
        other = time_to_tol("mixed", other_mode, timing=0)
        ms_this = ms / args.steps
        compare = {"form": forms[args.coarse], "ms_to_tol": ms_this, "iters": iters[-1],
                   "plain_fp64_ms_to_tol": plain["ms"], "plain_fp64_iters": plain["iters"],
                   "speedup_vs_plain_fp64": plain["ms"] / ms_this,
                   "rel_maxnorm_diff_UN_vs_plain_fp64": rel(uN_mixed, plain["uN"]),
                   "plain_fp64_unknown_updates_per_s": plain["ups"], "plain_fp64_fp64_pipe": fp64_pipe,
                   "variant": {"form": forms[other_mode], "coarse": other_mode, "ms_to_tol": other["ms"],
                               "iters": other["iters"], "speedup_vs_plain_fp64": plain["ms"] / other["ms"],
                               "rel_maxnorm_diff_UN_vs_plain_fp64": rel(other["uN"], plain["uN"])}}
        if cfg.get("src_t") is None:
            # common reference: the same parareal solve with half the fine step (s -> 2 s); the FIE
            # steps are first order in delta t (Sec. 2.2), so 2 |U_N(dt) - U_N(dt/2)| estimates the
            # temporal error of every arm at dt
            ref = time_to_tol("mixed", "fp64", s_fine=2 * cfg["s"], reps=1, timing=0)
            t_err = 2.0 * rel(plain["uN"], ref["uN"])
            gap = rel(uN_mixed, plain["uN"])
            accuracy = {"reference": f"parareal with FP32 fine line solves and s = {2 * cfg['s']} (half the fine "
                                     f"step), tol {cfg['tol']}",
                        "temporal_error_estimate_rel": t_err,
                        "rel_err_vs_reference": {"plain_fp64": rel(plain["uN"], ref["uN"]),
                                                 "this_form": rel(uN_mixed, ref["uN"]),
                                                 "variant": rel(other["uN"], ref["uN"])},
                        "fp32_gap_vs_plain_fp64_rel": gap,
                        "fp32_gap_over_temporal_error": gap / t_err if t_err > 0 else None}

    if args.fine == "dr":
        # Parareal/FIE-DR beside Parareal/FIE-FIE on the same workload and GPU (Sec. 4 pairs both)
        ms_fie, it_fie, uN_fie = time_fie_fie_to_tol(ps, torch, cfg, u0, stream)
        uN_dr = prob.state(cfg["N"]).cpu().numpy()
        compare = {"fie_dr_ms_to_tol": ms / args.steps, "fie_dr_iters": iters[-1],
                   "fie_fie_ms_to_tol": ms_fie, "fie_fie_iters": it_fie,
                   "rel_maxnorm_diff_UN_dr_vs_fie": float(np.abs(uN_dr - uN_fie).max() /
                                                          max(np.abs(uN_fie).max(), 1e-300))}

    cpu = None
    if rank == 0 and ws == 1 and args.cpu_seconds > 0:
        import oracle as orc
        orc.build()
        cpu = cpu_sample(cfg, args.cpu_seconds, args.fine)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
                "dominant_kernel_note": ("FP64 sweeps are bound by the FP64 issue rate (1.19 TFLOP/s measured)"
                                         if args.precision == "fp64" else None),
                "config": config_of(args, cfg), "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
                "roofline": roof, "cpu_baseline": cpu, "time_to_tol": compare, "accuracy": accuracy,
                "parareal_iterations": iters, "kernels": kernels,
                "autotune": ({"seconds_all_problems": AUTOTUNE["seconds"],
                              "chosen": [r[0] for r in tuned if r[2]],
                              "record_ms": {r[0]: round(r[1], 4) for r in tuned}}
                             if AUTOTUNE["on"] else None)}
        if "exact" in cfg:
            # the scalability experiment: error of the final iterate against the manufactured solution,
            # measured like Sec. 5 (max over the coarse times of the h-weighted 2-norm)
            h = 1.0 / (cfg["n"][0] + 1)
            err = max(float(np.sqrt(h * h * np.sum((prob.state(j).cpu().numpy() - cfg["exact"](j * cfg["T"] / cfg["N"]))
                                                   ** 2))) for j in range(1, cfg["N"] + 1))
            line["error_vs_exact_after_5_iterations"] = err
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
