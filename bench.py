#!/usr/bin/env python
"""Benchmark of one projection time step on the paper-shaped bubbly duct.

Workload: 224 x 224 x 640 cells (32.1M; the paper's "32 million control
volumes", Section 4 / abstract), 864 gas spheres of diameter 12h placed by
seeded rejection sampling, 1/7-power mean profile at Re_b = 5300 plus 8%
divergence-free perturbations, gravity along -z; synthetic inputs only.

A step is one call of the library's `step` (predictor terms, VOF advection,
curvature and surface force, pressure solve to rtol, projection). Timed with
CUDA events on the library's stream between barriers; the inputs (257 MB per
field) are larger than the 126 MB L2, so no flush is needed between steps.

Output: one JSON line (rank 0). With --impl reference the same metric is
measured for the FP64 CPU oracle on a bounded sample of the workload.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-steps/s & Poisson cell-updates/s at 32M cells; served p50/p99 vs FP64"
UNIT = "time-steps/s"
WORKLOAD = "paper-shaped duct 224x224x640 (32.1M cells), 864 spheres d=12h, Re_b=5300 1/7 profile + 8% noise"

# Algorithmic bytes per fine-grid cell for one launch of each kernel class:
# what the kernel must read and write at minimum.
# FP64 path (separate red and black launches, stored FP64 face coefficients):
#  smooth_l0   one colour: other-colour x (4), all face betas (24), own-colour
#              right side (4), own-colour x written (4)              = 36
#  restrict_l0 residual of 8 children averaged: x, f (16), betas (24),
#              coarse f written (1)                                  = 41
#  prolong_l0  fine x read and written (16), coarse x (1)            = 17
# Mixed path (FP32 V-cycle, finest level from the FP16 cell density, one
# launch per whole red-black sweep, x ping-ponged between two buffers):
#  smooth_l0   full sweep: old x (4), density (2), f (4), new x (4) = 14;
#              the first pre-smoothing sweep starts from zero (10); with
#              nu sweeps before and after: (10 + 14 (2 nu - 1)) / (2 nu)
#  restrict_l0 x, density, f (10), coarse f written (0.5)           = 10.5
#  prolong_l0  fine x read and written (8), coarse x (0.5)          = 8.5
#  residual_l0 FP64 outer residual (P 8, b 8, betas 24, FP32 r 4)   = 44
NU = 2


def algo_bytes_per_cell(cls: str, precision: str) -> float:
    if precision == "fp64":
        return {"smooth_l0": 36.0, "restrict_l0": 41.0, "prolong_l0": 17.0,
                "residual_l0": 40.0}[cls]
    # finest-level sweeps per cycle: one from zero (density 2, f 4, x out 4),
    # 2 NU - 2 from x (+ old x 4), and the last one, which also reads q for
    # the Krylov dots (+ 4)
    return {"smooth_l0": (10.0 + 14.0 * (2 * NU - 2) + 18.0) / (2 * NU), "restrict_l0": 10.5,
            "prolong_l0": 8.5, "residual_l0": 44.0}[cls]


KERNEL_SOURCE = {"fp64": {"smooth_l0": "k_mg.cu", "residual_l0": "k_poisson.cu",
                          "restrict_l0": "k_mg.cu", "prolong_l0": "k_mg.cu"},
                 "mixed": {"smooth_l0": "k_smooth_tma.cu", "residual_l0": "k_poisson.cu",
                           "restrict_l0": "k_smooth_tma.cu", "prolong_l0": "k_mg.cu"}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--nz", type=int, default=640, help="z cells (smaller for quick runs)")
    ap.add_argument("--graph", default="auto", choices=["auto", "cycle", "off"],
                    help="solver graph mode: auto captures the whole mixed solve (its loops "
                         "as conditional graph nodes); cycle replays only the V-cycle with the "
                         "loops on the host: the same kernels in the same order, and the mode "
                         "ncu can profile (it cannot profile kernel nodes of graphs with "
                         "conditional nodes)")
    ap.add_argument("--mg-tail", type=int, default=0,
                    help="coarse levels: 0 one launch per operation (replayed from the cycle's "
                         "graph), 1 one cluster launch per visit, 2 one grid-wide cooperative "
                         "launch per visit")
    ap.add_argument("--mg-tune", default="auto", choices=["auto", "off"],
                    help="launch shapes of the coarse levels' colour passes: timed when a "
                         "context is created (auto) or built in (off); the same bits either way")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-one-thread", action="store_true",
                    help="also time the oracle's sample on one host thread (slow)")
    ap.add_argument("--no-regular-array", action="store_true",
                    help="skip the 6x6x24 regular-array variant of the workload")
    ap.add_argument("--no-small-configs", action="store_true",
                    help="skip the static bubble (32^3, 20 steps) and the 64x64x128 swarm "
                         "(200 steps, FP64 against mixed)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--cpu-full-steps", type=int, default=0,
                    help="only time this many oracle steps on the whole 224x224x640 duct and "
                         "print them (slow: minutes per step)")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests in the serving run (0 skips it)")
    ap.add_argument("--ensemble-cases", type=int, default=64,
                    help="cases in the ensemble run (0 skips it)")
    ap.add_argument("--ensemble-profile-step", default=None, choices=["auto", "cycle"],
                    help="only build the ensemble of --ensemble-cases cases (graph option auto "
                         "or cycle), take three steps and bracket a fourth with "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# Multi-GPU: every rank advances an independent replica (its own seeded duct);
# the job's time is the slowest rank's, and the value counts every rank's steps.
_T0 = time.perf_counter()


def progress(what: str) -> None:
    """One line per finished part of the run on stderr (the JSON line stays
    the only output on stdout)."""
    print(f"[bench {time.perf_counter() - _T0:8.1f} s] {what}", file=sys.stderr, flush=True)


def replica_seed(rank: int) -> int:
    return 2106 + rank


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the ranks of the process group (x itself when dist
    is None); device is where the reduction tensor lives (cuda for NCCL, cpu
    for gloo)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, ms_max: float) -> float:
    """time-steps/s of the whole job: every rank's steps over the slowest rank's time."""
    return world * steps / (ms_max / 1e3)


# ----------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_for(cls: str, precision: str):
    """DRAM bytes per launch from the committed ncu table (profiles/
    ncu_traffic.txt: class, source file, its sha256, bytes per launch), or
    None when the kernel's source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        f = line.split()
        if len(f) != 4 or f[0] != cls or line.startswith("#"):
            continue
        if f[1] != KERNEL_SOURCE[precision][cls]:
            continue
        src = os.path.join(ROOT, "paper_2104_01636_b300", "csrc", f[1])
        if not os.path.exists(src):
            return None
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        return float(f[3]) if h == f[2] else None
    return None


# ----------------------------------------------------------------------------
def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


FULL_CELLS = 224 * 224 * 640


def sample_planes(steps: int, warmup: int) -> int:
    """z-planes of the oracle's bounded sample (the full 224 x 224 cross
    section): 16 while the reference arm's warmup + steps samples fit in
    about 3 minutes on the host (25 samples of ~8 s), fewer (even, at least
    8) for longer runs. Both CPU legs of a run use the same sample, so they
    report the same thing."""
    n = steps + warmup
    if n <= 25:
        return 16
    return max(8, 2 * ((16 * 25) // (2 * n)))


def cpu_baseline(args, steps=1, label="bounded sample", nz_s=16, threads=0, warmup=0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    the same generator on 224 x 224 x nz_s (~0.8M cells for 16 planes).
    Returns the measured seconds per sample step and the steps/s scaled to
    the 32.1M-cell metric by the cell ratio. The oracle's Jacobi-CG needs
    more iterations on the full grid than on a slab, so the scaled rate
    overstates the oracle at full size; the full-size measurement is
    recorded separately (profiles/oracle_full_duct.json). threads > 0 caps
    the oracle's OpenMP threads."""
    import oracle
    from paper_2104_01636_b300 import inputs as I
    if threads > 0:
        oracle.set_num_threads(threads)
    nb = round(864 * nz_s / 640)
    case = I.paper_shaped(224, 224, nz_s, nbub=nb, seed=2106)
    g, ph = case.grid, case.phys
    state = case.state()
    for s in range(warmup):
        *state, rep, st = oracle.step(g, ph, *state, case.dt, s, rtol=args.rtol)
    t_tot, iters = 0.0, 0
    for s in range(warmup, warmup + steps):
        t0 = time.perf_counter()
        *state, rep, st = oracle.step(g, ph, *state, case.dt, s, rtol=args.rtol)
        t_tot += time.perf_counter() - t0
        iters += rep["iters"]
    sps_sample = steps / t_tot
    return {
        "value": sps_sample * g.ncells / FULL_CELLS,
        "unit": UNIT,
        "cores": oracle.num_threads(),
        "cpu_model": cpu_model(),
        "host_cores": os.cpu_count(),
        "kind": "oracle",
        "sample": (f"{steps} timed oracle step(s) (after {warmup} untimed) of the same generator "
                   f"on 224x224x{nz_s} ({g.ncells} cells, {nb} spheres), rtol {args.rtol:g}; "
                   f"value = measured sample steps/s x {g.ncells}/{FULL_CELLS} cells ({label})"),
        "sample_cells": g.ncells,
        "sample_s_per_step": t_tot / steps,
        "poisson_cell_updates_per_s": g.ncells * iters / t_tot,
        "jacobi_cg_iters_per_step": iters / steps,
    }


def oracle_full_record():
    """The oracle timed once on the whole 224 x 224 x 640 duct (2 steps on
    the GPU machine's host cores, bench.py --cpu-full-steps 2), as committed."""
    p = os.path.join(ROOT, "profiles", "oracle_full_duct.json")
    if not os.path.exists(p):
        return None
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return None


def cpu_full(args):
    """--cpu-full-steps N: N oracle steps on the whole paper-shaped duct
    (224 x 224 x 640, 864 spheres; about 10 GB of host memory), timed one by
    one. Prints one JSON line; slow (minutes per step), never part of the
    default run."""
    import oracle
    from paper_2104_01636_b300 import inputs as I
    case = I.paper_shaped(seed=2106)
    g, ph = case.grid, case.phys
    state = case.state()
    per, its = [], []
    for s in range(args.cpu_full_steps):
        t0 = time.perf_counter()
        *state, rep, st = oracle.step(g, ph, *state, case.dt, s, rtol=args.rtol)
        per.append(time.perf_counter() - t0)
        its.append(rep["iters"])
    rec = {"oracle_full": {
        "workload": WORKLOAD, "cells": g.ncells, "steps": len(per), "rtol": args.rtol,
        "s_per_step": per, "jacobi_cg_iters": its,
        "value": len(per) / sum(per), "unit": UNIT,
        "poisson_cell_updates_per_s": g.ncells * sum(its) / sum(per),
        "cores": oracle.num_threads(), "host_cores": os.cpu_count(), "cpu_model": cpu_model(),
        "command": f"python bench.py --cpu-full-steps {args.cpu_full_steps} --rtol {args.rtol:g}"}}
    print(json.dumps(rec), flush=True)


def run_reference(args, rank):
    if rank != 0:
        return
    # each step is one oracle step on the bounded sample of sample_planes();
    # the same sample as the bench arm's cpu_baseline
    nz_s = sample_planes(args.steps, args.warmup)
    t0 = time.perf_counter()
    cb = cpu_baseline(args, steps=max(1, args.steps), label="reference arm", nz_s=nz_s,
                      warmup=args.warmup)
    wall = time.perf_counter() - t0
    line = {
        "impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # the measured time of one sample step (value scales it to 32.1M cells)
        "ms_per_step": 1e3 * cb["sample_s_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": cb["sample"],
                   "sample_cells": cb["sample_cells"]},
        "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "cpu_model", "kind",
                                            "sample")},
        "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "poisson_cell_updates_per_s": cb["poisson_cell_updates_per_s"],
        "jacobi_cg_iters_per_step": cb["jacobi_cg_iters_per_step"],
        "wall_s": wall,
        "oracle_full_duct": oracle_full_record(),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
SERVE_BUDGET = 40 << 30
SERVE_SLOTS = 8


def serving_run(vd, reqs, precision: int, rate, seed: int = 2108, rtol: float = 1e-8):
    """Submits the request mix to a VofServer with exponential inter-arrival
    gaps at `rate` requests/s (None: all at once, the saturation run) and
    returns latency percentiles (submit -> result) and throughput. Host
    copies of the inputs are made before the arrivals start."""
    import numpy as np
    gaps = (np.zeros(len(reqs)) if rate is None else
            np.random.default_rng(seed).exponential(1.0 / rate, len(reqs)))
    bufs = []
    for r in reqs:
        if r.kind == "step":
            bufs.append([np.array(a, dtype=np.float64, order="C", copy=True)
                         for a in r.case.state()])
        else:
            bufs.append([r.case.alpha.copy(), r.b.copy(), np.zeros_like(r.b)])
    sv = vd.c_solver(precision, rtol=rtol, max_iter=500)
    with vd.VofServer(SERVE_BUDGET, SERVE_SLOTS) as S:
        ids = []
        t0 = time.perf_counter()
        t_next = 0.0
        for r, gap, b in zip(reqs, gaps, bufs):
            t_next += gap
            delay = t0 + t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            c = r.case
            if r.kind == "step":
                ids.append(S.submit_step(c.grid, c.phys, sv, b, r.n_steps, c.dt))
            else:
                ids.append(S.submit_solve(c.grid, c.phys, sv, *b))
        res = [S.wait(i) for i in ids]
    bad = [x["status"] for x in res if x["status"] != "VOF_OK"]
    lat = np.array([x["t_finish"] - x["t_submit"] for x in res])
    span = max(x["t_finish"] for x in res) - min(x["t_submit"] for x in res)
    busy = sum(x["t_finish"] - x["t_admit"] for x in res)
    cell_steps = sum(r.case.grid.ncells * max(r.n_steps, 1) for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "requests_per_s": len(reqs) / span, "cell_steps_per_s": cell_steps / span,
            "mean_concurrency": busy / span, "failed": bad,
            "offered_rate": rate}


def serving(vd, I, n_req: int, do_fp64: bool):
    """Continuous-batching serving of a seeded ensemble mix: per precision a
    saturation run (all requests at once) gives the throughput, then Poisson
    arrivals at 70% of that throughput give p50/p99 latency."""
    reqs = I.serving_mix(n_req, seed=2108)
    serving_run(vd, reqs[:4], vd.PREC_MIXED_FP32, None)  # warm-up: modules, memory pool
    out = {"requests": n_req, "budget_bytes": SERVE_BUDGET, "slots": SERVE_SLOTS,
           "mix": ("grids {32^3, 64x64x128, 96x96x192, 128x128x256}, 1-64 spheres "
                   "d in [8,14]h, 50% STEP(1-10 steps) / 50% SOLVE, rtol 1e-8, seed 2108"),
           "load": "Poisson arrivals at 0.7 x the saturation throughput"}
    for name, prec in (("mixed", vd.PREC_MIXED_FP32), ("fp64", vd.PREC_FP64)):
        if name == "fp64" and not do_fp64:
            continue
        sat = serving_run(vd, reqs, prec, None)
        progress(f"serving {name} saturated run done")
        loaded = serving_run(vd, reqs, prec, 0.7 * sat["requests_per_s"])
        progress(f"serving {name} loaded run done")
        out[name] = {"saturation": sat, "loaded": loaded}
    return out


def ensemble_profile_step(vd, I, n_cases: int, graph: str, streams: int = 16):
    """The bench's ensemble, three steps, then one step between
    cudaProfilerStart and cudaProfilerStop; prints that step's host time."""
    import numpy as np
    import torch
    cases = I.ensemble_cases(n_cases, dims=(48, 48, 96), seed=2109)
    gm = {"auto": vd.GRAPH_AUTO, "cycle": vd.GRAPH_CYCLE}[graph]
    sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-8, max_iter=500, graph=gm)
    fields = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in c.state()] for c in cases]
    torch.cuda.synchronize()
    with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], sv, n_streams=streams,
                        mode=vd.VofEnsemble.BATCHED) as E:
        dts = [c.dt for c in cases]
        for s in range(3):
            E.step(fields, dts, s)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        t0 = time.perf_counter()
        E.step(fields, dts, 3)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"ensemble_profile_step": {"cases": n_cases, "graph": graph, "ms": ms}}))


def ensemble(vd, I, n_cases: int, streams: int = 16, steps: int = 5, warmup: int = 2,
             tune: int = 0):
    """n independent 48x48x96 ducts (4-16 spheres each, seeded) advanced
    together, fields resident on the device; mixed precision, rtol 1e-8.
    Timed on the host clock around whole ensemble steps (each call returns
    when every case has finished): batched solves with the whole step one
    graph launch and with the loops on the host, the cases overlapped on
    streams, and on one stream."""
    import numpy as np
    import torch
    cases = I.ensemble_cases(n_cases, dims=(48, 48, 96), seed=2109)
    out = {"cases": n_cases, "grid": "48x48x96", "cells_per_case": cases[0].grid.ncells,
           "precision": "mixed", "rtol": 1e-8, "steps": steps}
    # batched: the whole ensemble step one CUDA graph launch; batched_host_loops:
    # the same batched solve with its loops on the host
    runs = (("batched", streams, vd.VofEnsemble.BATCHED, vd.GRAPH_AUTO),
            ("batched_host_loops", streams, vd.VofEnsemble.BATCHED, vd.GRAPH_CYCLE),
            ("streams", streams, vd.VofEnsemble.STREAMS, vd.GRAPH_AUTO),
            ("one_stream", 1, vd.VofEnsemble.STREAMS, vd.GRAPH_AUTO))
    for label, ns, mode, graph in runs:
        sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-8, max_iter=500, graph=graph,
                         mg_tune=tune)
        fields = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in c.state()]
                  for c in cases]
        torch.cuda.synchronize()
        with vd.VofEnsemble(cases[0].grid, [c.phys for c in cases], sv, n_streams=ns,
                            mode=mode) as E:
            dts = [c.dt for c in cases]
            for s in range(warmup):
                E.step(fields, dts, s)
            torch.cuda.synchronize()
            n0 = E.launch_count()
            ph0 = E.phase_ms()
            g0 = E.graph_steps()
            t0 = time.perf_counter()
            for s in range(warmup, warmup + steps):
                reps = E.step(fields, dts, s, reports=True)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / steps
            launches = (E.launch_count() - n0) / steps
            graph_steps = (E.graph_steps() - g0) / steps
            phases = [(b - a) / steps for a, b in zip(ph0, E.phase_ms())]
            batched = E.batched
            shapes = mg_shapes(vd, E) if batched else None
        del fields
        progress(f"ensemble {label} timed")
        out[label] = {"n_streams": ns, "batched_solves": batched,
                      "ms_per_ensemble_step": ms,
                      "case_steps_per_s": n_cases / (ms / 1e3),
                      "cell_steps_per_s": n_cases * cases[0].grid.ncells / (ms / 1e3),
                      "kernel_launches_per_ensemble_step": launches,
                      "graph_launches_per_ensemble_step": graph_steps,
                      "ms_before_solve_solve_after": phases,
                      "max_inner_iters": max(r["iters"] for r in reps),
                      "mean_inner_iters": sum(r["iters"] for r in reps) / len(reps)}
        if shapes is not None:
            out[label]["mg_shapes"] = shapes
    return out


TUNE = {"auto": 0, "off": 1}


def mg_shapes(vd, obj):
    """The coarse levels' launch shapes of a context or of an ensemble's
    batched solve, by level."""
    out = {}
    for level in range(1, 16):
        try:
            sh = obj.mg_shape(level)
        except vd.VofError:
            continue
        out[str(level)] = {"planes_per_thread": sh[0], "block": sh[1], "restrict_block": sh[2],
                           "timed": sh[3]}
    return out


# ----------------------------------------------------------------------------
def small_configs(vd, I):
    """The two small configurations on the GPU, fields resident on the device:
    the static bubble (32^3, R = 8h, 20 steps, FP64 at rtol 1e-10) with exact
    and height-function curvature, reporting the pressure jump against the
    Laplace value 2 sigma / R and the spurious currents; and the rising swarm
    (64x64x128, 8 spheres, 200 steps) on the FP64 and the mixed path at rtol
    1e-8, reporting time per step and the mixed path's difference from FP64."""
    import numpy as np
    import torch
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def run(case, sv, steps):
        T = [dev(x) for x in case.state()]
        torch.cuda.synchronize()
        reps = []
        stream = torch.cuda.Stream()  # capturable: the solver replays its graphs
        with torch.cuda.stream(stream):
            with vd.VofContext(case.grid, case.phys, sv, stream=stream) as C:
                C.step(*T, case.dt, 0)  # the first step captures the graphs
                stream.synchronize()
                t0 = time.perf_counter()
                for s in range(1, steps):
                    reps.append(C.step(*T, case.dt, s))
                stream.synchronize()
                ms = (time.perf_counter() - t0) * 1e3 / max(steps - 1, 1)
        return [t.cpu().numpy() for t in T], reps, ms

    out = {}
    for name, km in (("exact_curvature", 1), ("height_function", 0)):
        case = I.static_bubble(kappa_mode=km)
        st, reps, ms = run(case, vd.c_solver(vd.PREC_FP64, rtol=1e-10, max_iter=400), 20)
        g, R, c = case.grid, case.radius, case.centres[0]
        x = (np.arange(g.nx) + 0.5) * g.h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        a, P = st[0], st[7]
        dp = P[(a < 1e-9) & (r < R - 2 * g.h)].mean() - P[(a > 1 - 1e-9) & (r > R + 2 * g.h)].mean()
        dpl = 2 * case.phys.sigma / R
        out.setdefault("static_bubble", {"grid": "32^3", "radius": "8h", "steps": 20,
                                         "laplace_pa": dpl})[name] = {
            "dp_over_laplace": dp / dpl, "max_u": reps[-1]["max_u"],
            "capillary_number": case.phys.mu_l * reps[-1]["max_u"] / case.phys.sigma,
            "ms_per_step": ms}
    case = I.rising_swarm(64, 64, 128, nbub=8, d_cells=12, seed=2104, steps=200)
    sw = {"grid": "64x64x128", "spheres": 8, "steps": 200, "rtol": 1e-8}
    states = {}
    for name, prec in (("fp64", vd.PREC_FP64), ("mixed", vd.PREC_MIXED_FP32)):
        st, reps, ms = run(case, vd.c_solver(prec, rtol=1e-8, max_iter=500), 200)
        states[name] = st
        sw[name] = {"ms_per_step": ms, "pcg_iters_per_step": float(np.mean([r["iters"] for r in reps])),
                    "max_div_dt": max(r["max_div"] for r in reps) * case.dt}
    f, m = states["fp64"], states["mixed"]
    vel = lambda s: np.concatenate([np.ravel(t) for t in s[1:7]])
    sw["mixed_vs_fp64"] = {
        "velocity_rel_l2": float(np.linalg.norm(vel(m) - vel(f)) / np.linalg.norm(vel(f))),
        "alpha_max_abs": float(np.abs(m[0] - f[0]).max()),
        "volume_rel_diff": float(abs(m[0].sum() - f[0].sum()) / f[0].sum())}
    out["rising_swarm"] = sw
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.cpu_full_steps > 0:
        if rank == 0:
            cpu_full(args)
        return

    import numpy as np
    import torch

    import paper_2104_01636_b300 as vd
    from paper_2104_01636_b300 import inputs as I

    torch.cuda.set_device(local)
    if args.ensemble_profile_step:
        if rank == 0:
            ensemble_profile_step(vd, I, args.ensemble_cases, args.ensemble_profile_step)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    nbub = round(864 * args.nz / 640)
    case = I.paper_shaped(224, 224, args.nz, nbub=nbub, seed=replica_seed(rank))
    g = case.grid
    N = g.ncells
    prec = vd.PREC_FP64 if args.precision == "fp64" else vd.PREC_MIXED_FP32
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gmode = {"auto": vd.GRAPH_AUTO, "cycle": vd.GRAPH_CYCLE, "off": vd.GRAPH_OFF}[args.graph]
        ctx = vd.VofContext(g, case.phys,
                            vd.c_solver(prec, rtol=args.rtol, max_iter=500, graph=gmode,
                                        mg_tail=args.mg_tail, mg_tune=TUNE[args.mg_tune]),
                            stream=stream)
        shapes = mg_shapes(vd, ctx)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        T = [dev(x) for x in case.state()]
        torch.cuda.synchronize()
        for s in range(args.warmup):
            ctx.step(*T, case.dt, s)
        barrier()

        # ---- timed region: device-resident inputs --------------------------
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        n0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = 0
        barrier()
        e0.record(stream)
        for s in range(args.warmup, args.warmup + args.steps):
            rep = ctx.step(*T, case.dt, s)
            iters += rep["iters"]
        e1.record(stream)
        barrier()
        launches = ctx.launch_count() - n0
        ck = clocks.stop()
        ms = e0.elapsed_time(e1)
        ms_max = max_over_ranks(ms, dist, "cuda")
        ms_per_step = ms_max / args.steps
        value = whole_job_rate(world, args.steps, ms_max)

        # ---- roofline: per-kernel CUDA events on the library stream --------
        ctx.set_timing(True)
        ctx.kernel_times()
        k_steps = max(2, min(args.steps, 5))
        solve_ms, it2 = 0.0, 0
        for s in range(k_steps):
            rep = ctx.step(*T, case.dt, args.warmup + args.steps + s)
            solve_ms += rep["ms"][4]
            it2 += rep["iters"]
        kt = ctx.kernel_times()
        ctx.set_timing(False)
        cls = max(KERNEL_SOURCE[args.precision], key=lambda k: kt.get(k, (0.0, 0))[0])
        kms, kn = kt[cls]
        avg_ms = kms / max(kn, 1)
        algo = algo_bytes_per_cell(cls, args.precision) * N
        peak, peak_kind = peaks()
        achieved = algo / (avg_ms / 1e3) / 1e9
        step_ms_timed = sum(v[0] for v in kt.values()) / k_steps
        roofline = {"bound": "hbm", "kernel": cls, "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic_for(cls, args.precision), "algorithmic_bytes": algo,
                    "avg_launch_ms": avg_ms, "launches_per_step": kn / k_steps,
                    # the kernel's time per step over the timed step (ms_per_step)
                    "share_of_step": kms / k_steps / ms_per_step,
                    "share_of_timed_classes": (kms / k_steps / step_ms_timed
                                               if step_ms_timed else None),
                    "classes_ms_per_step": {k: round(v[0] / k_steps, 4) for k, v in kt.items()}}
        poisson = N * it2 / (solve_ms / 1e3) if solve_ms > 0 else None
        solves = k_steps / (solve_ms / 1e3) if solve_ms > 0 else None

        progress("device-resident steps timed")
        # ---- end to end: the state in pinned host memory, copied in and out
        # every step by the host-buffer step of the C ABI (vof_step_host) --
        H = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in T]
        for h, t in zip(H, T):
            h.copy_(t)
        torch.cuda.synchronize()
        h2d = sum(t.numel() * t.element_size() for t in T)
        base = args.warmup + args.steps + k_steps
        ctx.step_host(*H, case.dt, base, report=False)  # allocates the device copy
        torch.cuda.synchronize()
        barrier()
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for s in range(args.steps):
            ctx.step_host(*H, case.dt, base + 1 + s, report=False)
        ctx.host_join()  # the last step's copies out
        e3.record(stream)
        barrier()
        ms_e2e = e2.elapsed_time(e3)
        e2e_value = whole_job_rate(world, args.steps, max_over_ranks(ms_e2e, dist, "cuda"))
        ctx.close()

        progress("host-buffer steps timed")
        # ---- the FP64 path on the same workload, for comparison ------------
        fp64 = None
        if args.precision == "mixed" and not args.no_fp64_compare:
            ctx64 = vd.VofContext(g, case.phys, vd.c_solver(vd.PREC_FP64, rtol=args.rtol,
                                                            max_iter=500), stream=stream)
            T64 = [dev(x) for x in case.state()]
            for s in range(2):
                ctx64.step(*T64, case.dt, s)
            n64 = max(1, min(args.steps, 5))
            it64 = 0
            barrier()
            e0.record(stream)
            for s in range(2, 2 + n64):
                it64 += ctx64.step(*T64, case.dt, s)["iters"]
            e1.record(stream)
            barrier()
            ms64 = e0.elapsed_time(e1)
            fp64 = {"value": n64 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64 / n64,
                    "pcg_iters_per_step": it64 / n64, "steps": n64, "rtol": args.rtol}
            ctx64.close()
            del T64

        progress("FP64 path timed")
        # ---- the paper's regular 6 x 6 x 24 bubble array (same grid) -------
        regular = None
        if not args.no_regular_array:
            rcase = I.paper_shaped(224, 224, args.nz, regular=True)
            ctxr = vd.VofContext(g, rcase.phys, vd.c_solver(prec, rtol=args.rtol, max_iter=500),
                                 stream=stream)
            TR = [dev(x) for x in rcase.state()]
            for s in range(2):
                ctxr.step(*TR, rcase.dt, s)
            nr = max(1, min(args.steps, 10))
            itr = 0
            barrier()
            e0.record(stream)
            for s in range(2, 2 + nr):
                itr += ctxr.step(*TR, rcase.dt, s)["iters"]
            e1.record(stream)
            barrier()
            msr = e0.elapsed_time(e1)
            regular = {"value": nr / (msr / 1e3), "unit": UNIT, "ms_per_step": msr / nr,
                       "pcg_iters_per_step": itr / nr, "steps": nr, "spheres": 864,
                       "layout": "regular 6 x 6 x 24 array (Section 4)"}
            ctxr.close()
            del TR

    progress("paper-shaped duct done")
    serve = None
    if world == 1 and args.serve_requests > 0:
        serve = serving(vd, I, args.serve_requests, not args.no_fp64_compare)
        progress("serving done")
    ens = None
    if world == 1 and args.ensemble_cases > 0:
        ens = ensemble(vd, I, args.ensemble_cases, tune=TUNE[args.mg_tune])
        progress("ensemble done")
    small = None
    if world == 1 and not args.no_small_configs:
        small = small_configs(vd, I)
        progress("small configurations done")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cb = None
    if world == 1 and not args.no_cpu_baseline:
        nz_s = sample_planes(args.steps, args.warmup)
        # three sample steps: 10-30 s of host work for the samples sample_planes() picks
        cb = cpu_baseline(args, steps=3, nz_s=nz_s)
        cb["oracle_full_duct"] = oracle_full_record()
        progress("CPU baseline done")
        if args.cpu_one_thread:
            one = cpu_baseline(args, steps=1, label="one host thread", nz_s=nz_s, threads=1)
            cb["one_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample",
                                                     "sample_s_per_step",
                                                     "poisson_cell_updates_per_s")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.nz == 640 else
                   f"paper-shaped duct 224x224x{args.nz} ({N / 1e6:.1f}M cells), {nbub} spheres "
                   "d=12h, Re_b=5300 1/7 profile + 8% noise",
                   "cells": N, "spheres": nbub, "rtol": args.rtol,
                   "precision": args.precision, "parallelism": f"replicas x{world}",
                   "graph": args.graph,
                   "l2": "inputs larger than L2 (257 MB per cell field), no flush",
                   "dt": case.dt},
        "poisson_cell_updates_per_s": poisson,
        "pcg_iters_per_step": iters / args.steps,
        "solves_per_s": solves,
        "roofline": roofline,
        "cpu_baseline": (None if cb is None else
                         {k: cb[k] for k in ("value", "unit", "cores", "cpu_model", "host_cores",
                                             "kind", "sample", "sample_cells",
                                             "sample_s_per_step", "poisson_cell_updates_per_s",
                                             "jacobi_cg_iters_per_step", "one_thread",
                                             "oracle_full_duct")
                          if k in cb}),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": h2d},
        "gpu_launches": launches,
        "mg_shapes": shapes,
        "clocks": ck,
        "fp64_path": fp64,
        "regular_array": regular,
        "serving": serve,
        "ensemble": ens,
        "small_configs": small,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
