"""Checkpoint/resume: a run interrupted, saved and resumed continues bit for
bit like the uninterrupted run (oracle on the CPU; the library on a GPU)."""
import os

import numpy as np
import pytest

import oracle
from paper_2104_01636_b300 import checkpoint as ck
from paper_2104_01636_b300 import inputs as I


def _case():
    return I.rising_swarm(20, 20, 24, nbub=2, seed=31, steps=4)


def test_roundtrip_and_header(tmp_path):
    case = _case()
    p = str(tmp_path / "c.bin")
    ck.save(p, case.grid, case.phys, case.state(), step_index=7, dt=case.dt, seed=31)
    hdr, arrs = ck.load(p)
    assert hdr["step_index"] == 7 and hdr["seed"] == 31 and hdr["dt"] == case.dt
    g, ph = ck.grid_phys(hdr)
    assert g == case.grid and ph == case.phys
    for a, b in zip(arrs, case.state()):
        assert np.array_equal(a, b)
    with open(p, "r+b") as f:  # a truncated file is refused
        f.truncate(os.path.getsize(p) - 8)
    with pytest.raises(ValueError):
        ck.load(p)


def test_oracle_resume_is_bitwise_identical(tmp_path):
    case = _case()
    g, ph = case.grid, case.phys
    s = case.state()
    for k in range(4):
        *s, rep, st = oracle.step(g, ph, *s, case.dt, k, rtol=1e-10)
    full = s
    s = case.state()
    for k in range(2):
        *s, rep, st = oracle.step(g, ph, *s, case.dt, k, rtol=1e-10)
    p = str(tmp_path / "mid.bin")
    ck.save(p, g, ph, s, step_index=2, dt=case.dt)
    hdr, s = ck.load(p)
    g2, ph2 = ck.grid_phys(hdr)
    for k in range(hdr["step_index"], 4):
        *s, rep, st = oracle.step(g2, ph2, *s, hdr["dt"], k, rtol=1e-10)
    for a, b in zip(s, full):
        assert np.array_equal(a, b)


@pytest.mark.gpu
def test_gpu_resume_is_bitwise_identical(tmp_path):
    import torch
    import paper_2104_01636_b300 as vd
    from gpu_util import dev, host
    case = _case()
    sv = vd.c_solver(1, rtol=1e-10, max_iter=300)
    with vd.VofContext(case.grid, case.phys, sv) as C:
        T = [dev(x) for x in case.state()]
        for k in range(4):
            C.step(*T, case.dt, k)
        full = [host(t) for t in T]
    p = str(tmp_path / "gpu.bin")
    with vd.VofContext(case.grid, case.phys, sv) as C:
        T = [dev(x) for x in case.state()]
        for k in range(2):
            C.step(*T, case.dt, k)
        ck.save(p, case.grid, case.phys, T, step_index=2, dt=case.dt, precision="mixed")
    hdr, arrs = ck.load(p)
    g, ph = ck.grid_phys(hdr)
    with vd.VofContext(g, ph, sv) as C:
        T = [dev(x) for x in arrs]
        for k in range(hdr["step_index"], 4):
            C.step(*T, hdr["dt"], k)
        torch.cuda.synchronize()
        for t, b in zip(T, full):
            assert np.array_equal(host(t), b)
