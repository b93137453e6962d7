"""Parity at the benchmark's full size: the paper-shaped duct of 224 x 224 x 640
cells (32.1M; 864 spheres of diameter 12h, 1/7-power profile with 8%
perturbations, seed 2106), in the configuration bench.py times (mixed
precision, rtol 1e-8, max_iter 500, default options, a context on a side
stream so the cycle is captured and replayed from a CUDA graph).

The local steps (operator, advection with its fluxes, face force, predictor)
are compared with the oracle element by element on the whole grid. The
pressure solve, which the oracle cannot finish at this size, is checked by a
property that holds at any size: its FP64 residual, evaluated on the host by
the oracle's operator, meets rtol. A whole step is checked for the
conservation of the liquid volume and for the solve's tolerance."""
import numpy as np
import pytest

import oracle
import paper_2104_01636_b300 as vd
from paper_2104_01636_b300 import inputs as I
from gpu_util import dev, host, rel_max

pytestmark = pytest.mark.gpu

NX, NY, NZ = 224, 224, 640


@pytest.fixture(scope="module")
def duct():
    return I.paper_shaped(NX, NY, NZ, nbub=864, seed=2106)


@pytest.fixture(scope="module")
def advected(duct):
    """The oracle's first advection step: alpha^{n+1}, fluxes, report."""
    return oracle.advect(duct.grid, duct.alpha, duct.u, duct.v, duct.w, duct.dt, 0, fluxes=True)


@pytest.fixture(scope="module")
def bench_ctx(duct):
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        C = vd.VofContext(duct.grid, duct.phys,
                          vd.c_solver(vd.PREC_MIXED_FP32, rtol=1e-8, max_iter=500), stream=stream)
    yield C, stream
    C.close()


def _sync(stream):
    stream.synchronize()


def test_operator_full_size(duct, bench_ctx):
    C, stream = bench_ctx
    g = duct.grid
    x = np.random.default_rng(7).normal(size=g.shapes()[0])
    bx, by, bz = oracle.beta(g, duct.phys, duct.alpha)
    ref = oracle.apply_A(g, bx, by, bz, x)
    import torch
    with torch.cuda.stream(stream):
        y = dev(np.zeros_like(x))
        C.vof_apply_operator(dev(duct.alpha), dev(x), y)
        _sync(stream)
    assert rel_max(host(y), ref) < 1e-12


def test_advection_full_size(duct, advected, bench_ctx):
    C, stream = bench_ctx
    g = duct.grid
    cs, us, vs, ws = g.shapes()
    a_o, fl_o, orep = advected
    import torch
    with torch.cuda.stream(stream):
        a = dev(duct.alpha)
        fl = [dev(np.zeros(s)) for s in (us, vs, ws)]
        rep = C.vof_advect(a, dev(duct.u), dev(duct.v), dev(duct.w), duct.dt, 0, fluxes=fl)
        _sync(stream)
    assert np.max(np.abs(host(a) - a_o)) < 1e-12
    for got, ref in zip(fl, fl_o):
        assert np.max(np.abs(host(got) - ref)) < 1e-13
    assert rep["vol_after"] == pytest.approx(orep["vol_after"], rel=1e-13)
    assert rep["vol_after"] == pytest.approx(rep["vol_before"], rel=1e-13)


def test_face_force_full_size(duct, bench_ctx):
    C, stream = bench_ctx
    g = duct.grid
    cs, us, vs, ws = g.shapes()
    ko, sxo, syo, szo, _ = oracle.ssf(g, duct.phys, duct.alpha)
    import torch
    with torch.cuda.stream(stream):
        k, sx, sy, sz = (dev(np.zeros(s)) for s in (cs, us, vs, ws))
        C.ssf_force(dev(duct.alpha), k, sx, sy, sz)
        _sync(stream)
    assert rel_max(host(k), ko) < 1e-12
    for got, ref in [(sx, sxo), (sy, syo), (sz, szo)]:
        assert rel_max(host(got), ref) < 1e-12


def test_predictor_full_size(duct, advected, bench_ctx):
    """Mixed path: the viscous term and the transport sum are FP32. The
    viscous term's rounding of the velocities is multiplied by
    dt mu_f / (h^2 rho) of up to ~0.1 in interface cells, where a liquid face
    viscosity meets a gas-dominated density; the transport sum is rounded to
    FP32 (6e-8 of itself) and divided by the cell's new density, which in such
    cells makes it of the order of the velocity itself. So the bound is FP32
    rounding on the velocity scale: 6e-8 of the largest velocity (measured
    1.2e-8)."""
    C, stream = bench_ctx
    g = duct.grid
    a1, fl, _ = advected
    ref_c = oracle.predict(g, duct.phys, duct.alpha, a1, duct.uc, duct.vc, duct.wc, duct.u,
                           duct.v, duct.w, *fl, duct.dt)
    ref_f = oracle.cell_to_face(g, *ref_c)
    import torch
    with torch.cuda.stream(stream):
        T = [dev(x) for x in (duct.uc, duct.vc, duct.wc, duct.u, duct.v, duct.w)]
        C.vof_predict(dev(duct.alpha), dev(a1), *T, *(dev(f) for f in fl), duct.dt)
        _sync(stream)
        got = [host(t) for t in T]
    for x, y in zip(got, list(ref_c) + list(ref_f)):
        assert np.max(np.abs(x - y)) < 6e-8 * np.max(np.abs(y))


def test_pressure_solve_full_size_meets_rtol(duct, advected, bench_ctx):
    """A seeded right side shaped like -div(u)/dt on the post-advection
    density; the residual b - A P is recomputed on the host in FP64 with the
    oracle's operator."""
    C, stream = bench_ctx
    g = duct.grid
    a1 = advected[0]
    rng = np.random.default_rng(2110)
    b = rng.normal(size=g.shapes()[0]) / duct.dt
    b -= b.mean()
    import torch
    with torch.cuda.stream(stream):
        p = dev(np.zeros_like(b))
        rep = C.pressure_solve(dev(a1), dev(b), p)
        _sync(stream)
        P = host(p)
    bx, by, bz = oracle.beta(g, duct.phys, a1)
    r = b - oracle.apply_A(g, bx, by, bz, P)
    res = np.linalg.norm(r) / np.linalg.norm(b)
    assert rep["res"] <= 1e-8
    assert res <= 1e-8 * (1 + 1e-3)
    assert res == pytest.approx(rep["res"], rel=1e-3)
    assert abs(P.mean()) <= 1e-12 * np.abs(P).max()


def test_step_full_size_conserves_volume(duct, bench_ctx):
    """The first step starts from discretely solenoidal face velocities, so
    the liquid volume is kept to round-off; the second from the projected
    ones, whose divergence is of the order of the solver tolerance."""
    C, stream = bench_ctx
    import torch
    vol0 = float(np.sum(duct.alpha, dtype=np.float64))
    with torch.cuda.stream(stream):
        T = [dev(x) for x in duct.state()]
        rep0 = C.step(*T, duct.dt, 0)
        _sync(stream)
        a0 = host(T[0])
        rep1 = C.step(*T, duct.dt, 1)
        _sync(stream)
        a1 = host(T[0])
    for rep in (rep0, rep1):
        assert rep["res"] <= 1e-8
        assert abs(rep["vol_clipped"]) <= 1e-12 * rep["vol_before"]
    # the projection: the divergence of the new face velocities, recomputed
    # here in FP64, is the one the step reports, and it is at the solver's
    # tolerance (div u^{n+1} = -dt (b - A P) for the solve's residual)
    u, v, w = (host(t) for t in T[4:7])
    inv_h = 1.0 / duct.grid.h
    # the same operations in the same order as the step's reduction
    div = ((((u[:, :, 1:] - u[:, :, :-1]) + v[:, 1:, :]) - v[:, :-1, :]) +
           np.roll(w, -1, axis=0) - w) * inv_h
    dmax = np.abs(div).max()
    assert dmax == pytest.approx(rep1["max_div"], rel=1e-12)
    assert dmax * duct.dt < 1e-8
    assert float(np.sum(a0, dtype=np.float64)) == pytest.approx(vol0, rel=1e-12)
    assert float(np.sum(a1, dtype=np.float64)) == pytest.approx(vol0, rel=1e-9)
    assert a1.min() >= 0.0 and a1.max() <= 1.0
