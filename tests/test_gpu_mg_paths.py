"""The two finest-level forms of the mixed-precision V-cycle: coefficients
formed from the cell density by the TMA-staged fused sweep (grids with
nx % 4 == 0 and at least two levels) and stored FP32 face arrays (other
grids). Both must reach the FP64 tolerance, agree with the oracle, converge
in about as many iterations as the FP64 path and be deterministic."""
import numpy as np
import pytest

import oracle
from paper_2104_01636_b300 import inputs as I
from gpu_util import ctx, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _problem(dims, nbub, seed, d_cells=8.0):
    g = I.Grid(*dims)
    c = I.place_spheres(g, nbub, d_cells * g.h, seed, wall_gap=g.h)
    a = I.sphere_alpha(g, c, d_cells * g.h / 2)
    rng = np.random.default_rng(seed)
    Pstar = rng.normal(size=g.shapes()[0])
    Pstar -= Pstar.mean()
    ph = I.Phys()
    bx, by, bz = oracle.beta(g, ph, a)
    b = oracle.apply_A(g, bx, by, bz, Pstar)
    return g, ph, a, b, Pstar


def _solve(g, ph, a, b, **kw):
    with ctx(g, ph, **kw) as C:
        p = dev(np.zeros_like(b))
        rep = C.pressure_solve(dev(a), dev(b), p)
        return host(p), rep


@pytest.mark.parametrize("dims", [(64, 48, 64),    # density path, partial tiles in y
                                  (96, 40, 36),    # density path, ragged in x and y
                                  (66, 40, 32)])   # nx % 4 != 0: stored FP32 faces
@pytest.mark.parametrize("nu,cyc", [(1, 0), (2, 0), (3, 0), (2, 1)])
def test_mixed_paths_reach_fp64_tolerance(dims, nu, cyc):
    """cyc 0: W-cycle (default), 1: V-cycle."""
    g, ph, a, b, Pstar = _problem(dims, 4, 31)
    kw = dict(nu_pre=nu, nu_post=nu, mg_cycle=cyc)
    P64, r64 = _solve(g, ph, a, b, rtol=1e-12, precision=0, **kw)
    P32, r32 = _solve(g, ph, a, b, rtol=1e-12, precision=1, **kw)
    assert r32["res"] <= 1e-12
    assert r32["iters"] <= 1.5 * r64["iters"] + 6, (r32["iters"], r64["iters"])
    assert rel_l2(P32, Pstar) < 1e-8
    assert rel_l2(P32, P64) < 1e-8


def test_density_path_is_deterministic():
    g, ph, a, b, _ = _problem((128, 96, 64), 10, 41)
    P1, r1 = _solve(g, ph, a, b, rtol=1e-10, precision=1)
    P2, r2 = _solve(g, ph, a, b, rtol=1e-10, precision=1)
    assert r1["iters"] == r2["iters"]
    assert np.array_equal(P1, P2)


def test_density_path_matches_oracle_at_paper_ratio():
    """Air-water density ratio 833 with many bubbles on a 96 x 96 x 64 grid."""
    g, ph, a, b, _ = _problem((96, 96, 64), 12, 43, d_cells=12.0)
    bx, by, bz = oracle.beta(g, ph, a)
    Po, orep, st = oracle.solve(g, bx, by, bz, b, rtol=1e-11)
    assert st == 0
    P, rep = _solve(g, ph, a, b, rtol=1e-11, precision=1)
    assert rep["res"] <= 1e-11
    assert rel_l2(P, Po) < 1e-6


def test_w_cycle_needs_fewer_iterations_than_v():
    g, ph, a, b, _ = _problem((96, 96, 64), 12, 47, d_cells=12.0)
    _, rw = _solve(g, ph, a, b, rtol=1e-10, precision=1, mg_cycle=0)
    _, rv = _solve(g, ph, a, b, rtol=1e-10, precision=1, mg_cycle=1)
    assert rw["res"] <= 1e-10 and rv["res"] <= 1e-10
    assert rw["iters"] < rv["iters"]


def _solve_counted(g, ph, a, b, **kw):
    with ctx(g, ph, **kw) as C:
        p = dev(np.zeros_like(b))
        n0 = C.launch_count()
        rep = C.pressure_solve(dev(a), dev(b), p)
        return host(p), rep, C.launch_count() - n0


@pytest.mark.parametrize("tail", [1, 2])
@pytest.mark.parametrize("dims,kw", [((64, 48, 64), {}),                 # cluster tail from level 2
                                     ((128, 96, 64), {}),                # cluster tail from level 3
                                     ((64, 32, 32), {"mg_w_depth": 8}),  # W visits inside the tail
                                     ((64, 32, 32), {"mg_cycle": 1}),    # V-cycle
                                     ((88, 40, 32), {"nu_pre": 3, "nu_post": 3})])
def test_coarse_tail_equals_launch_per_operation(dims, kw, tail):
    """The coarse levels run as one launch per smoothing pass, restriction
    and coarsest solve (default) or, from a small level down, as one launch
    per visit: on one thread-block cluster from a level of at most 8192
    cells (tail 1), or cooperatively on every SM with grid-wide barriers
    from a level of at most 131072 cells (tail 2). Same cell arithmetic in
    the same order, so the same iterates bit for bit, with fewer launches."""
    g, ph, a, b, _ = _problem(dims, 4, 53)
    Pt, rt, nt = _solve_counted(g, ph, a, b, rtol=1e-10, precision=1, graph=1, mg_tail=tail,
                                **kw)
    Po, ro, no = _solve_counted(g, ph, a, b, rtol=1e-10, precision=1, graph=1, **kw)
    assert rt["res"] <= 1e-10 and ro["res"] <= 1e-10
    assert rt["iters"] == ro["iters"]
    assert np.array_equal(Pt, Po), rel_l2(Pt, Po)
    assert nt < no, (nt, no)


def test_fp16_coarse_coefficients_reach_fp64_tolerance():
    """On 128^3, level 1 (64^3 = 262144 cells) is large enough to smooth and
    restrict with FP16 copies of its face coefficients (stored over a power
    of two). The cycle still has a single operator per level, so the mixed
    solve reaches the FP64 tolerance in about the FP64 path's iterations and
    is deterministic. Air-water density ratio, 16 bubbles of 12 cells."""
    g, ph, a, b, Pstar = _problem((128, 128, 128), 16, 59, d_cells=12.0)
    P64, r64 = _solve(g, ph, a, b, rtol=1e-11, precision=0)
    P32, r32 = _solve(g, ph, a, b, rtol=1e-11, precision=1)
    P32b, r32b = _solve(g, ph, a, b, rtol=1e-11, precision=1)
    assert r32["res"] <= 1e-11
    assert r32["iters"] <= 1.5 * r64["iters"] + 6, (r32["iters"], r64["iters"])
    assert rel_l2(P32, Pstar) < 1e-6
    assert rel_l2(P32, P64) < 1e-6
    assert r32b["iters"] == r32["iters"] and np.array_equal(P32, P32b)
