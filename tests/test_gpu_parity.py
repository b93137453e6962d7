"""GPU parity: the CUDA library against the FP64 CPU oracle, step by step and
for whole time steps, through the C ABI.

Tolerances (FP64 both sides; they differ only in rounding order, FMA use and
in the plane-constant algorithm, analytic on the GPU, bisection in the
oracle):
  * local kernels (operator, beta, predictor, face force, fluxes): a few
    hundred ulps of the field scale -> 1e-12 relative to max|field|;
  * volume fractions after advection: 1e-12 absolute per cell;
  * pressure solves at rtol 1e-12 on both sides: 1e-8 relative L2 (the
    residual tolerance times the operator's conditioning);
  * whole steps: |dp_gpu - dp_oracle| / dp_Laplace <= 1e-6 and velocity
    relative L2 <= 1e-8 after the stated number of steps.
"""
import numpy as np
import pytest

import oracle
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host, rel_l2, rel_max

pytestmark = pytest.mark.gpu

RAGGED = [(37, 21, 30), (32, 32, 32), (70, 12, 18)]


def _spheres(g, n, seed, d_cells=8.0):
    c = I.place_spheres(g, n, d_cells * g.h, seed, wall_gap=g.h)
    return c, I.sphere_alpha(g, c, d_cells * g.h / 2)


@pytest.mark.parametrize("dims", RAGGED)
def test_operator_parity(dims):
    g = I.Grid(*dims)
    ph = I.Phys()
    _, a = _spheres(g, 2, 3)
    x = np.random.default_rng(1).normal(size=g.shapes()[0])
    bx, by, bz = oracle.beta(g, ph, a)
    ref = oracle.apply_A(g, bx, by, bz, x)
    with ctx(g, ph) as C:
        y = dev(np.zeros_like(x))
        C.vof_apply_operator(dev(a), dev(x), y)
        assert rel_max(host(y), ref) < 1e-12


@pytest.mark.parametrize("dims", [(37, 21, 30), (48, 40, 64)])
def test_pressure_solve_parity(dims):
    g = I.Grid(*dims)
    ph = I.Phys()
    _, a = _spheres(g, 3, 4)
    rng = np.random.default_rng(2)
    Pstar = rng.normal(size=g.shapes()[0])
    Pstar -= Pstar.mean()
    bx, by, bz = oracle.beta(g, ph, a)
    b = oracle.apply_A(g, bx, by, bz, Pstar) + 3.0  # non-zero mean is removed
    Po, orep, st = oracle.solve(g, bx, by, bz, b, rtol=1e-12)
    assert st == 0
    with ctx(g, ph, rtol=1e-12) as C:
        p = dev(np.zeros_like(b))
        rep = C.pressure_solve(dev(a), dev(b), p)
        P = host(p)
    assert rep["res"] <= 1e-12 and rep["iters"] < 100
    assert rep["b_mean"] == pytest.approx(orep["b_mean"], rel=1e-10)
    assert abs(P.mean()) < 1e-12 * np.abs(P).max()
    assert rel_l2(P, Po) < 1e-8
    assert rel_l2(P, Pstar) < 1e-8


@pytest.mark.parametrize("dims,per", [((37, 21, 30), False), ((32, 24, 20), True)])
def test_advect_parity(dims, per):
    g = I.Grid(*dims, per_x=int(per), per_y=int(per))
    _, a0 = _spheres(I.Grid(*dims), 3, 5)
    u, v, w = I.curl_noise(I.Grid(*dims), 0.1, seed=6, kmax=3)
    w = w + 0.04
    dt = 0.45 * g.h / max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    a_o = a0.copy()
    with ctx(g, I.Phys()) as C:
        a_d = dev(a0)
        U, Vv, W = dev(u), dev(v), dev(w)
        for s in range(4):
            rep = C.vof_advect(a_d, U, Vv, W, dt, s)
            a_o, orep = oracle.advect(g, a_o, u, v, w, dt, s)
            assert np.max(np.abs(host(a_d) - a_o)) < 1e-12
            assert rep["vol_after"] == pytest.approx(orep["vol_after"], rel=1e-13)
            assert rep["vol_after"] == pytest.approx(rep["vol_before"], rel=1e-13)


def test_advect_unit_courant_translation_exact():
    g = I.Grid(20, 16, 24)
    c = np.array([[10.3 * g.h, 7.8 * g.h, 12.1 * g.h]])
    a0 = I.sphere_alpha(g, c, 5 * g.h)
    cs, us, vs, ws = g.shapes()
    with ctx(g, I.Phys()) as C:
        a = dev(a0)
        Z = [dev(np.zeros(us)), dev(np.zeros(vs)), dev(np.full(ws, 0.02))]
        for s in range(g.nz):
            C.vof_advect(a, *Z, g.h / 0.02, s, report=False)
        assert np.max(np.abs(host(a) - a0)) < 1e-12


@pytest.mark.parametrize("kappa_mode", [0, 1])
def test_ssf_force_parity(kappa_mode):
    g = I.Grid(40, 36, 48)
    ph = I.Phys(kappa_mode=kappa_mode, kappa_exact=1.0 / (4 * g.h))
    _, a = _spheres(g, 3, 7, d_cells=10)
    ko, sxo, syo, szo, orep = oracle.ssf(g, ph, a)
    cs, us, vs, ws = g.shapes()
    with ctx(g, ph) as C:
        k, sx, sy, sz = dev(np.zeros(cs)), dev(np.zeros(us)), dev(np.zeros(vs)), dev(np.zeros(ws))
        C.ssf_force(dev(a), k, sx, sy, sz)
        assert rel_max(host(k), ko) < 1e-12
        for got, ref in [(sx, sxo), (sy, syo), (sz, szo)]:
            assert rel_max(host(got), ref) < 1e-12
        assert np.array_equal(host(sx) != 0, sxo != 0)


@pytest.mark.parametrize("conv", [0, 1])
def test_predict_parity(conv):
    case = I.rising_swarm(36, 28, 40, nbub=3, seed=8, steps=1)
    g = case.grid
    ph = I.Phys(**{**case.phys.__dict__, "conv_scheme": conv})
    a1, _ = oracle.advect(g, case.alpha, case.u, case.v, case.w, case.dt, 0)
    ref = oracle.predict(g, ph, case.alpha, a1, case.u, case.v, case.w, case.dt)
    with ctx(g, ph) as C:
        U, Vv, W = dev(case.u), dev(case.v), dev(case.w)
        C.vof_predict(dev(case.alpha), dev(a1), U, Vv, W, case.dt)
        got = [host(U), host(Vv), host(W)]
    for x, y in zip(got, ref):
        assert rel_max(x, y) < 1e-12


def test_project_parity():
    case = I.rising_swarm(36, 28, 40, nbub=3, seed=9, steps=1)
    g, ph = case.grid, case.phys
    kap, sx, sy, sz, _ = oracle.ssf(g, ph, case.alpha)
    rng = np.random.default_rng(10)
    uh = case.u + 0.01 * rng.normal(size=case.u.shape)
    vh = case.v + 0.01 * rng.normal(size=case.v.shape)
    wh = case.w + 0.01 * rng.normal(size=case.w.shape)
    uo, vo, wo, Po, orep, st = oracle.project(g, ph, case.alpha, uh, vh, wh, case.P, sx, sy, sz,
                                              case.dt, rtol=1e-12)
    assert st == 0
    with ctx(case, rtol=1e-12) as C:
        U, Vv, W, P = dev(uh), dev(vh), dev(wh), dev(case.P)
        rep = C.project(dev(case.alpha), U, Vv, W, P, dev(sx), dev(sy), dev(sz), case.dt)
        assert rel_l2([host(U), host(Vv), host(W)], [uo, vo, wo]) < 1e-10
        assert rel_l2(host(P), Po) < 1e-8
        assert rep["max_div"] * case.dt < 1e-10


def _laplace_jump(case, a, P):
    g, R, c = case.grid, case.radius, case.centres[0]
    x = (np.arange(g.nx) + 0.5) * g.h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    return P[(a < 1e-9) & (r < R - 2 * g.h)].mean() - P[(a > 1 - 1e-9) & (r > R + 2 * g.h)].mean()


@pytest.mark.parametrize("kappa_mode", [1, 0])
def test_step_static_bubble_20_steps(kappa_mode):
    case = I.static_bubble(kappa_mode=kappa_mode)
    g, ph = case.grid, case.phys
    ao, uo, vo, wo, Po = case.alpha, case.u, case.v, case.w, case.P
    with ctx(case, rtol=1e-12) as C:
        T = [dev(x) for x in (case.alpha, case.u, case.v, case.w, case.P)]
        for s in range(20):
            rep = C.step(*T, case.dt, s)
            ao, uo, vo, wo, Po, orep, st = oracle.step(g, ph, ao, uo, vo, wo, Po, case.dt, s,
                                                      rtol=1e-12)
            assert st == 0
        a, u, v, w, P = (host(t) for t in T)
    dp_l = 2 * ph.sigma / case.radius
    dp, dpo = _laplace_jump(case, a, P), _laplace_jump(case, ao, Po)
    assert abs(dp - dpo) / dp_l <= 1e-6
    if kappa_mode == 1:
        assert dp == pytest.approx(dp_l, rel=1e-9)
        assert rep["max_u"] < 1e-11
    else:
        assert rel_l2([u, v, w], [uo, vo, wo]) <= 1e-8
        assert rep["max_u"] == pytest.approx(orep["max_u"], rel=1e-6)
    assert np.max(np.abs(a - ao)) < 1e-12


def test_step_rising_swarm_parity():
    case = I.rising_swarm(32, 32, 48, nbub=3, seed=11, steps=6)
    g, ph = case.grid, case.phys
    ao, uo, vo, wo, Po = case.alpha, case.u, case.v, case.w, case.P
    with ctx(case, rtol=1e-12) as C:
        T = [dev(x) for x in (case.alpha, case.u, case.v, case.w, case.P)]
        for s in range(case.steps):
            rep = C.step(*T, case.dt, s)
            ao, uo, vo, wo, Po, orep, st = oracle.step(g, ph, ao, uo, vo, wo, Po, case.dt, s,
                                                      rtol=1e-12)
            assert st == 0
            assert rep["vol_after"] == pytest.approx(orep["vol_after"], rel=1e-13)
        a, u, v, w, P = (host(t) for t in T)
    assert rel_l2([u, v, w], [uo, vo, wo]) <= 1e-8
    assert np.max(np.abs(a - ao)) < 1e-10
    assert rel_l2(P, Po) < 1e-7
