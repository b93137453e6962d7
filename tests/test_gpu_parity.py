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
    relative L2 <= 1e-8 after the stated number of steps. The Laplace jump
    is a difference of two region means of P and inherits the solve's
    residual times the operator's conditioning (~1e5 here): the oracle
    against itself at rtol 1e-12 vs 1e-14 already differs by 9e-6 dp_L, so
    the static-bubble runs use rtol 1e-13 on both sides (2e-7 dp_L).
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


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims", [(37, 21, 30), (48, 40, 64)])
def test_pressure_solve_parity(dims, prec):
    """FP64 and mixed (FP32 V-cycle, FP64 residual/updates) solves both reach
    rtol 1e-12 and agree with the oracle to the conditioning bound."""
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
    with ctx(g, ph, rtol=1e-12, precision=prec) as C:
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
    cs, us, vs, ws = g.shapes()
    with ctx(g, I.Phys()) as C:
        a_d = dev(a0)
        U, Vv, W = dev(u), dev(v), dev(w)
        fl = [dev(np.zeros(s_)) for s_ in (us, vs, ws)]
        for s in range(4):
            rep = C.vof_advect(a_d, U, Vv, W, dt, s, fluxes=fl)
            a_o, flo, orep = oracle.advect(g, a_o, u, v, w, dt, s, fluxes=True)
            assert np.max(np.abs(host(a_d) - a_o)) < 1e-12
            for x, y in zip(fl, flo):
                assert np.max(np.abs(host(x) - y)) < 1e-13
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
@pytest.mark.parametrize("prec", [0, 1])
def test_predict_parity(conv, prec):
    """FP64 path: 1e-12 of the field. The mixed path forms the viscous term
    and the transport sum in FP32: its error is FP32 rounding of parts of the
    step's increment, so it is bounded by 1e-6 of the largest increment
    u_hat - u^n."""
    case = I.rising_swarm(36, 28, 40, nbub=3, seed=8, steps=1)
    g = case.grid
    ph = I.Phys(**{**case.phys.__dict__, "conv_scheme": conv})
    a1, fl, _ = oracle.advect(g, case.alpha, case.u, case.v, case.w, case.dt, 0, fluxes=True)
    ref_c = oracle.predict(g, ph, case.alpha, a1, case.uc, case.vc, case.wc, case.u, case.v,
                           case.w, *fl, case.dt)
    ref_f = oracle.cell_to_face(g, *ref_c)
    with ctx(g, ph, precision=prec) as C:
        T = [dev(x) for x in (case.uc, case.vc, case.wc, case.u, case.v, case.w)]
        C.vof_predict(dev(case.alpha), dev(a1), *T, *(dev(f) for f in fl), case.dt)
        got = [host(t) for t in T]
    before = (case.uc, case.vc, case.wc, case.u, case.v, case.w)
    for x, y, x0 in zip(got, list(ref_c) + list(ref_f), before):
        if prec == 0:
            assert rel_max(x, y) < 1e-12
        else:
            assert np.max(np.abs(x - y)) < 1e-6 * np.max(np.abs(y - x0))


def test_project_parity():
    case = I.rising_swarm(36, 28, 40, nbub=3, seed=9, steps=1)
    g, ph = case.grid, case.phys
    kap, sx, sy, sz, _ = oracle.ssf(g, ph, case.alpha)
    rng = np.random.default_rng(10)
    uhc, vhc, whc = (x + 0.01 * rng.normal(size=x.shape) for x in (case.uc, case.vc, case.wc))
    uh, vh, wh = oracle.cell_to_face(g, uhc, vhc, whc)
    *ref, Po, orep, st = oracle.project(g, ph, case.alpha, uhc, vhc, whc, uh, vh, wh, case.P,
                                        sx, sy, sz, case.dt, rtol=1e-12)
    assert st == 0
    with ctx(case, rtol=1e-12) as C:
        T = [dev(x) for x in (uhc, vhc, whc, uh, vh, wh)]
        P = dev(case.P)
        rep = C.project(dev(case.alpha), *T, P, dev(sx), dev(sy), dev(sz), case.dt)
        assert rel_l2([host(t) for t in T], ref) < 1e-10
        assert rel_l2(host(P), Po) < 1e-8
        assert rep["max_div"] * case.dt < 1e-10


def _laplace_jump(case, a, P):
    g, R, c = case.grid, case.radius, case.centres[0]
    x = (np.arange(g.nx) + 0.5) * g.h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
    return P[(a < 1e-9) & (r < R - 2 * g.h)].mean() - P[(a > 1 - 1e-9) & (r > R + 2 * g.h)].mean()


def _run_both(case, steps, rtol, precision=0):
    g, ph = case.grid, case.phys
    ref = case.state()
    reps, oreps = [], []
    with ctx(case, rtol=rtol, precision=precision) as C:
        T = [dev(x) for x in case.state()]
        for s in range(steps):
            reps.append(C.step(*T, case.dt, s))
            *ref, orep, st = oracle.step(g, ph, *ref, case.dt, s, rtol=rtol)
            assert st == 0
            oreps.append(orep)
        got = [host(t) for t in T]
    return got, ref, reps, oreps


@pytest.mark.parametrize("kappa_mode", [1, 0])
def test_step_static_bubble_20_steps(kappa_mode):
    case = I.static_bubble(kappa_mode=kappa_mode)
    got, ref, reps, oreps = _run_both(case, 20, rtol=1e-13)
    dp_l = 2 * case.phys.sigma / case.radius
    dp, dpo = _laplace_jump(case, got[0], got[7]), _laplace_jump(case, ref[0], ref[7])
    assert abs(dp - dpo) / dp_l <= 1e-6
    if kappa_mode == 1:
        assert dp == pytest.approx(dp_l, rel=1e-9)
        assert reps[-1]["max_u"] < 1e-11
    else:
        assert rel_l2(got[1:7], ref[1:7]) <= 1e-8
        assert reps[-1]["max_u"] == pytest.approx(oreps[-1]["max_u"], rel=1e-6)
    assert np.max(np.abs(got[0] - ref[0])) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_step_rising_swarm_parity(prec):
    case = I.rising_swarm(32, 32, 48, nbub=3, seed=11, steps=6)
    got, ref, reps, oreps = _run_both(case, case.steps, rtol=1e-12, precision=prec)
    for r, o in zip(reps, oreps):
        assert r["vol_after"] == pytest.approx(o["vol_after"], rel=1e-13)
    assert rel_l2(got[1:7], ref[1:7]) <= 1e-8
    assert np.max(np.abs(got[0] - ref[0])) < 1e-10
    assert rel_l2(got[7], ref[7]) < 1e-7


@pytest.mark.parametrize("prec", [0, 1])
def test_step_single_phase_duct_parity(prec):
    """No bubble: alpha is 1 everywhere, so the interface lists are empty and
    the surface force is zero; the step is the single-phase projection of the
    laminar duct flow with noise. alpha stays 1 to rounding (each sweep's
    flux difference and divergence term cancel to an ulp), as in the oracle.
    Mixed path: both solves reach 1e-13, and P differs from the oracle's by
    what the predictor's FP32 increments (about 1e-8 of u_hat) put into the
    right side, about 1.5e-6 Pa on a pressure that falls to 2.5 Pa when only
    the noise drives it: 3e-7 relative, hence the bar of 1e-6."""
    case = I.rising_swarm(32, 32, 48, nbub=0, seed=5, steps=3)
    got, ref, reps, oreps = _run_both(case, case.steps, rtol=1e-12, precision=prec)
    assert np.max(np.abs(got[0] - 1.0)) < 1e-13
    assert np.max(np.abs(got[0] - ref[0])) < 1e-13
    assert rel_l2(got[1:7], ref[1:7]) <= (1e-11 if prec == 0 else 1e-8)
    assert rel_l2(got[7], ref[7]) < (1e-9 if prec == 0 else 1e-6)
    for r in reps:
        assert r["max_div"] * case.dt < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_step_ragged_grid_parity(prec):
    """A grid that fills no tile evenly (40 x 24 x 50: 32 x 32 sweep tiles,
    32 x 8 cell tiles and z chunks all ragged; an odd-width level, 5 x 3 x
    ..., in the hierarchy) with two small bubbles: whole steps against the
    oracle."""
    case = I.rising_swarm(40, 24, 50, nbub=2, d_cells=8, seed=13, steps=3)
    got, ref, reps, oreps = _run_both(case, case.steps, rtol=1e-12, precision=prec)
    for r, o in zip(reps, oreps):
        assert r["vol_after"] == pytest.approx(o["vol_after"], rel=1e-13)
    assert rel_l2(got[1:7], ref[1:7]) <= (1e-10 if prec == 0 else 1e-8)
    assert np.max(np.abs(got[0] - ref[0])) < (1e-12 if prec == 0 else 1e-10)
