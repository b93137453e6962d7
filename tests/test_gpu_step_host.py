"""The host-buffer step (vof_step_host): the state lives in host memory, is
copied in and out by the library around and during the step, and the result
is bitwise that of step() on device arrays. Covers pinned and pageable host
memory, the FP64 and mixed paths, a context on the legacy default stream and
one on a side stream (captured solve), several steps in a row with and
without reports (the pipelined loop, completed by vof_host_join), and an
error (CFL) that leaves the context usable."""
import numpy as np
import pytest
import torch

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _device_steps(case, sv, stream, steps):
    T = [dev(a) for a in case.state()]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, sv, stream=stream) as C:
            reps = [C.step(*T, case.dt, s) for s in steps]
    torch.cuda.synchronize()
    return [host(t) for t in T], reps


def _host_steps(case, sv, stream, steps, pinned, report=True):
    H = [torch.from_numpy(np.array(a, dtype=np.float64, order="C", copy=True)) for a in case.state()]
    if pinned:
        H = [h.pin_memory() for h in H]
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, sv, stream=stream) as C:
            reps = [C.step_host(*H, case.dt, s, report=report) for s in steps]
            if not report:  # the last call's copies out may still be running
                C.host_join()
            stream.synchronize()
    return [h.numpy().copy() for h in H], reps


@pytest.mark.parametrize("prec", [vd.PREC_FP64, vd.PREC_MIXED_FP32])
@pytest.mark.parametrize("side_stream", [False, True])
def test_step_host_equals_device_step(prec, side_stream):
    case = I.rising_swarm(48, 40, 64, nbub=4, d_cells=9, seed=95, steps=3)
    sv = vd.c_solver(prec, rtol=1e-9, max_iter=300)
    stream = torch.cuda.Stream() if side_stream else torch.cuda.default_stream()
    ref, rr = _device_steps(case, sv, stream, range(3))
    got, rg = _host_steps(case, sv, stream, range(3), pinned=True)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    for a, b in zip(rg, rr):
        assert a["iters"] == b["iters"] and a["res"] == b["res"]
        assert a["vol_after"] == b["vol_after"] and a["max_div"] == b["max_div"]


@pytest.mark.parametrize("side_stream", [False, True])
def test_step_host_pipelined_loop(side_stream):
    """Calls without a report: each call's copies in overlap the previous
    call's copies out; after host_join and a synchronisation the host state
    is bitwise that of device steps."""
    case = I.rising_swarm(48, 40, 64, nbub=4, d_cells=9, seed=99, steps=4)
    sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-9, max_iter=300)
    stream = torch.cuda.Stream() if side_stream else torch.cuda.default_stream()
    ref, _ = _device_steps(case, sv, stream, range(4))
    got, _ = _host_steps(case, sv, stream, range(4), pinned=True, report=False)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_step_host_two_solves():
    """The paper's two pressure solves per step (p~ kept in the context):
    P is copied out after the two solutions are combined."""
    case = I.rising_swarm(40, 32, 48, nbub=3, d_cells=8, seed=100, steps=3)
    sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-9, max_iter=300, ssf_solves=2)
    stream = torch.cuda.Stream()
    ref, rr = _device_steps(case, sv, stream, range(3))
    got, rg = _host_steps(case, sv, stream, range(3), pinned=True)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert [r["iters"] for r in rg] == [r["iters"] for r in rr]


def test_step_host_pageable_memory():
    case = I.rising_swarm(40, 32, 48, nbub=3, d_cells=8, seed=96, steps=2)
    sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-9, max_iter=300)
    stream = torch.cuda.Stream()
    ref, _ = _device_steps(case, sv, stream, range(2))
    got, _ = _host_steps(case, sv, stream, range(2), pinned=False)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_step_host_cfl_error_then_usable():
    """A time step over the CFL limit is refused before anything runs; the
    same context then steps normally from the unchanged host state."""
    case = I.rising_swarm(40, 32, 48, nbub=3, d_cells=8, seed=97, steps=1)
    sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-9, max_iter=300)
    stream = torch.cuda.Stream()
    ref, _ = _device_steps(case, sv, stream, [0])
    H = [torch.from_numpy(np.array(a, dtype=np.float64, order="C", copy=True)).pin_memory()
         for a in case.state()]
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, sv, stream=stream) as C:
            with pytest.raises(vd.VofError) as ei:
                C.step_host(*H, 1e6 * case.dt, 0)
            assert ei.value.name == "VOF_ERR_CFL"
            stream.synchronize()
            for h, a in zip(H, case.state()):
                assert np.array_equal(h.numpy(), a)
            C.step_host(*H, case.dt, 0)
            stream.synchronize()
    for h, b in zip(H, ref):
        assert np.array_equal(h.numpy(), b)


def test_step_host_rejects_device_tensors():
    case = I.rising_swarm(32, 32, 32, nbub=1, d_cells=8, seed=98, steps=1)
    with vd.VofContext(case.grid, case.phys, vd.c_solver(vd.PREC_MIXED_FP32)) as C:
        T = [dev(a) for a in case.state()]
        with pytest.raises(TypeError):
            C.step_host(*T, case.dt, 0)


def test_step_host_copies_stay_inside_the_host_arrays():
    """Every host array sits inside a larger pinned buffer whose margins hold
    a canary: the copies in and out read and write exactly the fields."""
    case = I.rising_swarm(40, 32, 48, nbub=3, d_cells=8, seed=103, steps=2)
    sv = vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-9, max_iter=300)
    stream = torch.cuda.Stream()
    ref, _ = _device_steps(case, sv, stream, range(2))
    guard, canary = 4096, -12345.6789
    bigs, views = [], []
    for a in case.state():
        big = torch.full((a.size + 2 * guard,), canary, dtype=torch.float64).pin_memory()
        big[guard:guard + a.size] = torch.from_numpy(np.ascontiguousarray(a).ravel())
        bigs.append(big)
        views.append(big[guard:guard + a.size].view(a.shape))
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, sv, stream=stream) as C:
            for s in range(2):
                C.step_host(*views, case.dt, s, report=False)
            C.host_join()
            stream.synchronize()
    for big, view, r in zip(bigs, views, ref):
        assert bool((big[:guard] == canary).all()) and bool((big[-guard:] == canary).all())
        assert np.array_equal(view.numpy(), r)
