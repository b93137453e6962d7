"""Pins of the oracle's PLIC geometry and height-function curvature.

Each test checks the oracle against something other than itself: exact
rational volumes, symmetry, brute-force counting, the symbolic curvature of
a surface, and the closed-form curvature of spheres and cylinders.
"""
import math
from fractions import Fraction
from itertools import product

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2104_01636_b300.inputs import Grid, sphere_alpha


def exact_halfspace_volume(m, a, lo=(0, 0, 0), hi=(1, 1, 1)):
    """Exact volume of {x in box : m.x <= a} in rational arithmetic, by
    inclusion-exclusion over the box vertices (negative components are
    reflected, zero components contribute their extent)."""
    a = Fraction(a)
    pos, ext = [], Fraction(1)
    for mi, l, u in zip(m, lo, hi):
        mi, l, u = Fraction(mi), Fraction(l), Fraction(u)
        if mi == 0:
            ext *= u - l
        elif mi > 0:
            pos.append((mi, l, u))
        else:
            a -= mi * (l + u)
            pos.append((-mi, l, u))
    n = len(pos)
    if n == 0:
        return ext * (1 if a >= 0 else 0)
    tot = Fraction(0)
    for v in product((0, 1), repeat=n):
        t = a - sum(mi * (u if vi else l) for (mi, l, u), vi in zip(pos, v))
        if t > 0:
            tot += (-1) ** sum(v) * t ** n
    den = math.factorial(n)
    for mi, _, _ in pos:
        den *= mi
    return ext * tot / den


def _dyadic(rng, scale, n):
    return [float(np.round(rng.uniform(-scale, scale) * 1024) / 1024) for _ in range(n)]


def test_plane_volume_matches_exact_rationals():
    rng = np.random.default_rng(1)
    worst = 0.0
    for t in range(400):
        m = _dyadic(rng, 1.0, 3)
        if t % 7 == 0:
            m[t % 3] = 0.0  # axis-parallel planes
        if t % 11 == 0:
            m[(t + 1) % 3] = 2.0 ** -30  # nearly degenerate normals
        lo = sum(min(x, 0) for x in m)
        hi = sum(max(x, 0) for x in m)
        a = float(np.round(rng.uniform(lo - 0.05, hi + 0.05) * 4096) / 4096)
        exact = exact_halfspace_volume([Fraction(x) for x in m], Fraction(a))
        got = oracle.plane_volume(m, a)
        worst = max(worst, abs(got - float(exact)))
    assert worst < 2e-15, worst


def test_plane_volume_special_cases():
    # corner simplex a^3 / (6 m1 m2 m3)
    m = [0.25, 0.5, 0.75]
    assert oracle.plane_volume(m, 0.125) == pytest.approx(0.125 ** 3 / (6 * 0.25 * 0.5 * 0.75), rel=1e-14)
    # the diagonal plane through the cube centre halves it
    assert oracle.plane_volume([1, 1, 1], 1.5) == pytest.approx(0.5, abs=1e-15)
    # axis-aligned planes: V = a / m
    assert oracle.plane_volume([0, 0, 2.0], 0.5) == pytest.approx(0.25, abs=1e-15)
    assert oracle.plane_volume([0, -2.0, 0], -0.5) == pytest.approx(0.75, abs=1e-15)
    assert oracle.plane_volume([0, 0, 0], 0.0) == 1.0
    assert oracle.plane_volume([0, 0, 0], -1e-300) == 0.0


def test_plane_volume_complement_symmetry():
    rng = np.random.default_rng(2)
    for _ in range(200):
        m = rng.normal(size=3)
        a = rng.uniform(-2, 2)
        assert oracle.plane_volume(m, a) + oracle.plane_volume(-m, -a) == pytest.approx(1.0, abs=2e-15)


def test_plane_volume_brute_force():
    n = 96
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    for m, a in [([0.3, -0.5, 0.2], -0.05), ([0.7, 0.1, 0.2], 0.4), ([-0.2, -0.3, -0.5], -0.8)]:
        frac = np.mean(m[0] * X + m[1] * Y + m[2] * Z <= a)
        assert abs(oracle.plane_volume(m, a) - frac) < 3.0 / n


def test_plane_constant_roundtrip():
    rng = np.random.default_rng(3)
    for t in range(300):
        m = rng.normal(size=3)
        if t % 5 == 0:
            m[t % 3] = 0.0
        alpha = rng.uniform(1e-9, 1 - 1e-9)
        d = oracle.plane_constant(m, alpha)
        assert abs(oracle.plane_volume(m, d) - alpha) < 1e-14
    # axis-aligned: d = alpha * m
    assert oracle.plane_constant([0, 0, 1.0], 0.3) == pytest.approx(0.3, abs=1e-15)


def test_normal_points_from_liquid_into_gas():
    g = Grid(8, 8, 12)
    a = np.zeros((12, 8, 8))
    a[:5] = 1.0
    a[5] = 0.4  # liquid below z = 5.4 h
    n = oracle.normal(g, a, 3, 4, 5)
    assert n[0] == 0.0 and n[1] == 0.0 and n[2] > 0.0
    # a 45-degree interface in (x, z): symmetric, so |n_x| = |n_z|
    a = np.zeros((12, 8, 8))
    for k in range(12):
        for i in range(8):
            a[k, :, i] = 1.0 if i + k < 9 else (0.5 if i + k == 9 else 0.0)
    n = oracle.normal(g, a, 4, 4, 5)
    assert n[0] > 0 and n[2] > 0 and n[1] == 0.0
    assert n[0] == pytest.approx(n[2], rel=1e-14)


def test_hf_direction_tie_break():
    assert oracle.hf_direction([1.0, 1.0 + 1e-12, 0.0]) == 0
    assert oracle.hf_direction([1.0, 1.1, 0.0]) == 1
    assert oracle.hf_direction([0.2, -0.3, 0.9]) == 2
    assert oracle.hf_direction([1.0, 1.0, 1.0]) == 0


def _sphere_kappa_errors(n, R_cells, gas=True):
    g = Grid(n, n, n)
    R = R_cells * g.h
    c = np.array([[n / 2 * g.h + 0.31 * g.h, n / 2 * g.h - 0.17 * g.h, n / 2 * g.h + 0.07 * g.h]])
    a = sphere_alpha(g, c, R, sub=32)
    if not gas:
        a = 1.0 - a
    kap, valid = oracle.curvature(g, a)
    sel = valid & (a > 1e-12) & (a < 1 - 1e-12)
    exact = 2.0 / R if gas else -2.0 / R
    return np.abs(kap[sel] / exact - 1.0), sel.sum()


def test_curvature_sphere_sign_and_convergence():
    e1, n1 = _sphere_kappa_errors(24, 6)
    e2, n2 = _sphere_kappa_errors(48, 12)
    assert n1 > 100 and n2 > 400
    assert np.mean(e1) < 0.05 and np.mean(e2) < 0.02
    assert np.mean(e2) < 0.5 * np.mean(e1)  # converges with resolution
    ed, _ = _sphere_kappa_errors(24, 6, gas=False)  # liquid drop: kappa = -2/R
    assert np.mean(ed) < 0.05


def test_curvature_cylinder():
    n, R_cells = 32, 9.0
    g = Grid(n, n, 8)
    R = R_cells * g.h
    # gas cylinder along z: exact alpha by 2-D sampling (z-invariant)
    s = 64
    off = (np.arange(s) + 0.5) / s
    xs = (np.arange(n)[:, None] + off[None, :]) * g.h - (n / 2 + 0.23) * g.h
    ys = (np.arange(n)[:, None] + off[None, :]) * g.h - (n / 2 - 0.11) * g.h
    inside = (xs[None, :, None, :] ** 2 + ys[:, None, :, None] ** 2) < R * R
    gas2 = inside.mean(axis=(2, 3))  # (ny, nx)
    a = np.broadcast_to(1.0 - gas2, (8, n, n)).copy()
    kap, valid = oracle.curvature(g, a)
    sel = valid & (a > 1e-12) & (a < 1 - 1e-12)
    assert sel.sum() > 50
    err = np.abs(kap[sel] * R - 1.0)
    assert np.mean(err) < 0.03


def test_curvature_quadric_matches_symbolic():
    """For a height function that is a quadratic in (x, y), the column sums
    are exact cell averages, so the scheme's derivatives are exact and the
    curvature must equal the surface's at the column centre."""
    X, Y = sp.symbols("x y")
    c = dict(z0=8.4, bx=0.21, by=-0.13, cxx=0.021, cxy=-0.012, cyy=0.015)  # cell units
    f = (c["z0"] + c["bx"] * X + c["by"] * Y + c["cxx"] * X ** 2 + c["cxy"] * X * Y +
         c["cyy"] * Y ** 2)
    nrm = sp.sqrt(1 + sp.diff(f, X) ** 2 + sp.diff(f, Y) ** 2)
    # unit normal pointing into the liquid (liquid below the surface)
    kappa_expr = sp.diff(sp.diff(f, X) / nrm, X) + sp.diff(sp.diff(f, Y) / nrm, Y)
    kfun = sp.lambdify((X, Y), kappa_expr, "numpy")
    ffun = sp.lambdify((X, Y), f, "numpy")
    n, nz = 14, 18
    g = Grid(n, n, nz, h=1.0)
    s = 200
    off = (np.arange(s) + 0.5) / s
    alpha = np.zeros((nz, n, n))
    ctr = n / 2
    for j in range(n):
        for i in range(n):
            xs = (i + off[:, None]) - ctr
            ys = (j + off[None, :]) - ctr
            H = ffun(xs, ys)
            for k in range(nz):
                alpha[k, j, i] = np.mean(np.clip(H - k, 0.0, 1.0))
    kap, valid = oracle.curvature(g, alpha)
    checked = 0
    for k in range(nz):
        for j in range(4, n - 4):
            for i in range(4, n - 4):
                if valid[k, j, i]:
                    ex = kfun(i + 0.5 - ctr, j + 0.5 - ctr)
                    assert kap[k, j, i] == pytest.approx(ex, rel=2e-3, abs=2e-5)
                    checked += 1
    assert checked >= 30
