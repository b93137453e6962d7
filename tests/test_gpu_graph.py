"""Contexts on a capturable stream replay captured CUDA graphs: the FP64
path its V-cycle, the mixed path its whole pressure solve, whose loops are
conditional WHILE nodes steered by device-side control kernels. Both give
bitwise the results of direct launches with host-driven loops (contexts on
the legacy default stream, which cannot be captured)."""
import numpy as np
import pytest
import torch

import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _run(case, solver, stream, nsteps):
    st = [dev(a) for a in case.state()]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, solver, stream=stream) as C:
            # the steps' launches (not the launch-shape timing at creation,
            # which only the first context of a shape runs)
            n0 = C.launch_count()
            reps = [C.step(*st, case.dt, s) for s in range(nsteps)]
            n = C.launch_count() - n0
    torch.cuda.synchronize()
    return [host(t) for t in st], reps, n


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_direct_launches(prec):
    case = I.rising_swarm(64, 48, 64, nbub=5, d_cells=10, seed=91, steps=3)
    sv = vd.c_solver(prec, rtol=1e-9, max_iter=300)
    direct, rd, nd = _run(case, sv, torch.cuda.default_stream(), 3)
    graph, rg, ng = _run(case, sv, torch.cuda.Stream(), 3)
    for a, b in zip(direct, graph):
        assert np.array_equal(a, b)
    assert [r["iters"] for r in rd] == [r["iters"] for r in rg]
    assert [r["refinements"] for r in rd] == [r["refinements"] for r in rg]
    assert [r["res"] for r in rd] == [r["res"] for r in rg]
    if prec == 0:
        assert nd == ng
    else:
        # the captured solve adds a control kernel per iteration and drops
        # the host loop's readback kernel per iteration
        assert abs(ng - nd) < 0.2 * nd


def _solve(case, solver, stream, b, p0=None):
    P = dev(np.zeros_like(b) if p0 is None else p0)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, solver, stream=stream) as C:
            try:
                rep, err = C.pressure_solve(dev(case.alpha), dev(b), P), None
            except vd.VofError as e:
                rep, err = e.report, e.name
    torch.cuda.synchronize()
    return host(P), rep, err


def test_captured_solve_zero_right_side_and_nonconvergence():
    case = I.rising_swarm(48, 32, 48, nbub=3, d_cells=8, seed=92, steps=1)
    rng = np.random.default_rng(5)
    # a right side that is constant: zero after its mean is removed
    b0 = np.full(case.alpha.shape, 3.0)
    for stream in (torch.cuda.default_stream(), torch.cuda.Stream()):
        P, rep, err = _solve(case, vd.c_solver(1, rtol=1e-10), stream, b0, rng.normal(size=b0.shape))
        assert err is None and rep["iters"] == 0 and not P.any()
    # a tolerance it cannot reach in 3 iterations: same error, same last iterate
    b = rng.normal(size=b0.shape)
    sv = vd.c_solver(1, rtol=1e-14, max_iter=3)
    Pd, rd, ed = _solve(case, sv, torch.cuda.default_stream(), b)
    Pg, rg, eg = _solve(case, sv, torch.cuda.Stream(), b)
    assert ed == eg == "VOF_ERR_NOT_CONVERGED"
    assert rd["iters"] == rg["iters"] == 3
    assert np.array_equal(Pd, Pg)


def test_captured_solves_alternate_between_two_graphs():
    """The two-solve mode solves into two pressures every step, and a solve
    into a new pointer is captured again: bitwise the host-driven results."""
    case = I.rising_swarm(48, 32, 48, nbub=3, d_cells=8, seed=93, steps=3)
    sv = vd.c_solver(1, rtol=1e-9, max_iter=300, ssf_solves=2)
    direct, rd, _ = _run(case, sv, torch.cuda.default_stream(), 3)
    graph, rg, _ = _run(case, sv, torch.cuda.Stream(), 3)
    for a, b in zip(direct, graph):
        assert np.array_equal(a, b)
    b = np.random.default_rng(6).normal(size=case.alpha.shape)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with vd.VofContext(case.grid, case.phys, vd.c_solver(1, rtol=1e-10), stream=stream) as C:
            outs = []
            for _ in range(3):  # three output pointers: each one is captured anew
                P = dev(np.zeros_like(b))
                C.pressure_solve(dev(case.alpha), dev(b), P)
                outs.append(host(P))
    torch.cuda.synchronize()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
