"""Duct driver: advance a case for many steps on the GPU with periodic
statistics samples and checkpoints, resume from a checkpoint, or restart a
laden run from an unladen one by inserting bubbles (Section 4: the laden
simulation starts from the fully developed unladen field with the bubbles
placed in it).

    python -m paper_2104_01636_b300.run --steps 200 --nz 64 --out run1
    python -m paper_2104_01636_b300.run --resume run1/ckpt.bin --steps 200 --out run2
    python -m paper_2104_01636_b300.run --insert-bubbles 86 --resume run1/ckpt.bin ...

Everything runs through the library (VofContext.step, VofStats); the state
stays on the device between steps.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import time

import numpy as np


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=224)
    ap.add_argument("--ny", type=int, default=224)
    ap.add_argument("--nz", type=int, default=640)
    ap.add_argument("--bubbles", type=int, default=864, help="spheres in a fresh case")
    ap.add_argument("--unladen", action="store_true", help="fresh case without bubbles")
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--stats-every", type=int, default=10)
    ap.add_argument("--ckpt-every", type=int, default=0, help="0: only at the end")
    ap.add_argument("--resume", default=None, help="checkpoint to continue from")
    ap.add_argument("--insert-bubbles", type=int, default=0,
                    help="with --resume: place this many spheres (d = 12h) into the field")
    ap.add_argument("--seed", type=int, default=2106)
    ap.add_argument("--out", default="run_out")
    return ap.parse_args(argv)


def initial_state(args):
    from paper_2104_01636_b300 import checkpoint as ck
    from paper_2104_01636_b300 import inputs as I
    if args.resume:
        header, arrs = ck.load(args.resume)
        grid, phys = ck.grid_phys(header)
        step0, dt = header["step_index"], header["dt"]
        if args.insert_bubbles > 0:
            d = 12 * grid.h
            centres = I.place_spheres(grid, args.insert_bubbles, d, args.seed)
            alpha = np.minimum(arrs[0], I.sphere_alpha(grid, centres, d / 2))
            arrs[0] = alpha
            phi = I.gas_fraction(alpha)
            phys = dataclasses.replace(phys, g_z=-I.GRAV,
                                       rho0=(1 - phi) * phys.rho_l + phi * phys.rho_g)
        return grid, phys, arrs, step0, dt
    nb = 0 if args.unladen else args.bubbles
    case = I.paper_shaped(args.nx, args.ny, args.nz, nbub=nb, seed=args.seed)
    return case.grid, case.phys, list(case.state()), 0, case.dt


def main(argv=None):
    args = parse(argv)
    import torch

    import paper_2104_01636_b300 as vd
    from paper_2104_01636_b300 import checkpoint as ck

    os.makedirs(args.out, exist_ok=True)
    grid, phys, arrs, step0, dt = initial_state(args)
    prec = vd.PREC_FP64 if args.precision == "fp64" else vd.PREC_MIXED_FP32
    stream = torch.cuda.Stream()
    T = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    torch.cuda.synchronize()
    log = open(os.path.join(args.out, "log.jsonl"), "a")
    with torch.cuda.stream(stream), \
            vd.VofContext(grid, phys, vd.c_solver(prec, rtol=args.rtol, max_iter=500),
                          stream=stream) as C, vd.VofStats(grid) as S:
        t0 = time.perf_counter()
        for s in range(step0, step0 + args.steps):
            rep = C.step(*T, dt, s)
            if args.stats_every and (s - step0) % args.stats_every == 0:
                S.accumulate(T[0], T[1], T[2], T[3], stream)
            log.write(json.dumps({"step": s, "iters": rep["iters"], "res": rep["res"],
                                  "max_div": rep["max_div"], "max_u": rep["max_u"],
                                  "vol": rep["vol_after"]}) + "\n")
            if args.ckpt_every and (s + 1 - step0) % args.ckpt_every == 0:
                stream.synchronize()
                ck.save(os.path.join(args.out, "ckpt.bin"), grid, phys, T, s + 1, dt,
                        seed=args.seed, precision=args.precision)
        stream.synchronize()
        wall = time.perf_counter() - t0
        ck.save(os.path.join(args.out, "ckpt.bin"), grid, phys, T, step0 + args.steps, dt,
                seed=args.seed, precision=args.precision)
        sums, n = S.sums()
        np.save(os.path.join(args.out, "stats_sums.npy"), sums)
    log.close()
    summary = {"steps": args.steps, "wall_s": wall, "steps_per_s": args.steps / wall,
               "stats_samples": n, "cells": grid.nx * grid.ny * grid.nz}
    with open(os.path.join(args.out, "summary.json"), "w") as f:
        json.dump(summary, f)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
