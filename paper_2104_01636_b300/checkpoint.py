"""Checkpoint and resume of the time-step state.

The paper restarts its laden run from the unladen run's final field
(Section 4) and integrates for about 1.5 million steps, so a run must be able
to stop and continue. A checkpoint is one raw little-endian binary file:

    magic   8 bytes  b"VOFCKPT1"
    header  JSON (utf-8), preceded by its length as uint64: grid, physical
            constants, step index, seed, precision, time step, array names
            and shapes
    arrays  float64, C order, in the header's order: alpha, uc, vc, wc,
            u, v, w, P

Resuming from a checkpoint reproduces the uninterrupted run bit for bit,
because the state is the whole input of the next step (the pressure is the
solver's initial guess).
"""
from __future__ import annotations

import dataclasses
import json
import os
import struct

import numpy as np

MAGIC = b"VOFCKPT1"
NAMES = ("alpha", "uc", "vc", "wc", "u", "v", "w", "P")


def save(path: str, grid, phys, state, step_index: int, dt: float, seed: int | None = None,
         precision: str = "fp64") -> None:
    """state: the eight arrays (numpy or torch, any device) in NAMES order."""
    arrs = []
    for a in state:
        if hasattr(a, "detach"):
            a = a.detach().cpu().numpy()
        arrs.append(np.ascontiguousarray(a, dtype="<f8"))
    header = {
        "grid": dataclasses.asdict(grid), "phys": dataclasses.asdict(phys),
        "step_index": int(step_index), "dt": float(dt), "seed": seed, "precision": precision,
        "arrays": [{"name": n, "shape": list(a.shape)} for n, a in zip(NAMES, arrs)],
    }
    hb = json.dumps(header, sort_keys=True).encode()
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<Q", len(hb)))
        f.write(hb)
        for a in arrs:
            f.write(a.tobytes(order="C"))
    os.replace(tmp, path)  # never leave a half-written checkpoint behind


def load(path: str):
    """Returns (header dict, list of the eight numpy arrays)."""
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a checkpoint")
        (n,) = struct.unpack("<Q", f.read(8))
        header = json.loads(f.read(n).decode())
        arrs = []
        for spec in header["arrays"]:
            shape = tuple(spec["shape"])
            count = int(np.prod(shape))
            buf = f.read(8 * count)
            if len(buf) != 8 * count:
                raise ValueError(f"{path}: truncated at {spec['name']}")
            arrs.append(np.frombuffer(buf, dtype="<f8").reshape(shape).copy())
    return header, arrs


def grid_phys(header):
    """Rebuild the grid and constants recorded in a header."""
    from paper_2104_01636_b300.inputs import Grid, Phys
    return Grid(**header["grid"]), Phys(**header["phys"])
