"""Pins of the oracle's viscous term (Eq. 2, the full stress
div(mu (grad u + grad u^T)); steps 8-10 with the face viscosity from the
linear averaging of step 10).

The term is read off the predictor with no transport and no body force:
rho^{n+1} u_hat = rho^n u + dt V with alpha unchanged. Each pin checks it
against something other than its own formula:

* constant mu, any quadratic velocity field: second-order central and
  two-point differences are exact on quadratics, so away from the walls the
  discrete term must equal mu (lap u + grad div u) of the polynomial to
  round-off (a wrong sign of the transposed part, or a tangential
  difference taken in the wrong direction or at the wrong cell, fails it);
* no-slip walls: a field odd about a wall plane has ghost values exactly
  minus the interior ones, so the same identity must hold in the cells next
  to each wall and in the corners (a wrong ghost sign on any component or
  tangential difference fails it);
* two fluids: the face fluxes telescope, so a field that vanishes near the
  walls feels no net viscous force for any viscosity field; and a shear
  layer whose discrete traction is the same on every face (mu jumping by
  55 across the interface) is in equilibrium cell by cell.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2104_01636_b300.inputs import Grid, Phys, sphere_alpha

X, Y, Z = sp.symbols("x y z")


def viscous(g, ph, alpha, q):
    """The oracle's viscous force per unit volume on every cell component."""
    cs, us, vs, ws = g.shapes()
    u0, v0, w0 = np.zeros(us), np.zeros(vs), np.zeros(ws)
    dt = 1.0
    out = oracle.predict(g, ph, alpha, alpha, *q, u0, v0, w0, u0, v0, w0, dt)
    rho = alpha * ph.rho_l + (1.0 - alpha) * ph.rho_g
    return [(o - qc) * rho / dt for o, qc in zip(out, q)]


def expected_full_stress(fields, mu):
    """mu (lap q_c + d_c div q) of polynomial fields, symbolically."""
    div = sum(sp.diff(f, s) for f, s in zip(fields, (X, Y, Z)))
    return [sp.expand(mu * (sp.diff(f, X, 2) + sp.diff(f, Y, 2) + sp.diff(f, Z, 2) +
                            sp.diff(div, s))) for f, s in zip(fields, (X, Y, Z))]


def sample(g, expr):
    f = sp.lambdify((X, Y, Z), expr, "numpy")
    x = (np.arange(g.nx) + 0.5) * g.h
    y = (np.arange(g.ny) + 0.5) * g.h
    z = (np.arange(g.nz) + 0.5) * g.h
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    return np.broadcast_to(np.asarray(f(Xg, Yg, Zg), dtype=np.float64), g.shapes()[0]).copy()


def _rand_quadratic(rng):
    mons = [1, X, Y, Z, X * X, Y * Y, Z * Z, X * Y, X * Z, Y * Z]
    return sum(sp.Float(rng.uniform(-1, 1)) * m for m in mons)


def _const_mu_phys(mu=0.7):
    return Phys(rho_l=1.0, rho_g=1.0, mu_l=mu, mu_g=mu)


def _check(g, ph, fields, sel):
    q = [sample(g, f) for f in fields]
    a = np.ones(g.shapes()[0])
    got = viscous(g, ph, a, q)
    exp = [sample(g, e) for e in expected_full_stress(fields, ph.mu_l)]
    scale = max(np.abs(e).max() for e in exp)
    assert scale > 0.1
    for gc, ec in zip(got, exp):
        assert np.max(np.abs(gc[sel] - ec[sel])) <= 1e-9 * scale


def test_interior_quadratic_fields_give_lap_plus_grad_div():
    g = Grid(9, 8, 10, h=0.37)
    rng = np.random.default_rng(41)
    fields = [_rand_quadratic(rng) for _ in range(3)]
    # the transposed part is not small for this field
    div = sum(sp.diff(f, s) for f, s in zip(fields, (X, Y, Z)))
    assert any(abs(float(sp.diff(div, s))) > 0.2 for s in (X, Y, Z))
    sel = np.zeros(g.shapes()[0], dtype=bool)
    sel[1:-1, 1:-1, 1:-1] = True  # no ghost, no wrap in z
    _check(g, _const_mu_phys(), fields, sel)


@pytest.mark.parametrize("wall", ["x0", "x1", "y0", "y1"])
def test_no_slip_ghosts_exact_for_fields_odd_about_the_wall(wall):
    g = Grid(8, 7, 9, h=0.5)
    Lx, Ly = g.nx * g.h, g.ny * g.h
    dist = {"x0": X, "x1": Lx - X, "y0": Y, "y1": Ly - Y}[wall]
    rng = np.random.default_rng({"x0": 1, "x1": 2, "y0": 3, "y1": 4}[wall])
    # distance to the wall times a linear function of the coordinates along
    # it: odd about the wall plane, zero on it (every component: no slip),
    # quadratic overall
    tang = (Y, Z) if wall[0] == "x" else (X, Z)  # coordinates along the wall
    fields = [dist * (sp.Float(rng.uniform(-1, 1)) + sp.Float(rng.uniform(-1, 1)) * tang[0] +
                      sp.Float(rng.uniform(-1, 1)) * tang[1]) for _ in range(3)]
    sel = np.zeros(g.shapes()[0], dtype=bool)
    if wall == "x0":
        sel[1:-1, 1:-1, 0:2] = True
    elif wall == "x1":
        sel[1:-1, 1:-1, -2:] = True
    elif wall == "y0":
        sel[1:-1, 0:2, 1:-1] = True
    else:
        sel[1:-1, -2:, 1:-1] = True
    _check(g, _const_mu_phys(), fields, sel)


@pytest.mark.parametrize("corner", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_no_slip_ghosts_exact_in_the_corners(corner):
    g = Grid(7, 6, 8, h=0.5)
    dx = X if corner[0] == 0 else g.nx * g.h - X
    dy = Y if corner[1] == 0 else g.ny * g.h - Y
    rng = np.random.default_rng(10 + 2 * corner[0] + corner[1])
    fields = [sp.Float(rng.uniform(0.5, 1.5)) * dx * dy for _ in range(3)]
    sel = np.zeros(g.shapes()[0], dtype=bool)
    ci = slice(0, 2) if corner[0] == 0 else slice(-2, None)
    cj = slice(0, 2) if corner[1] == 0 else slice(-2, None)
    sel[1:-1, cj, ci] = True
    _check(g, _const_mu_phys(), fields, sel)


def test_viscous_fluxes_telescope_for_any_viscosity_field():
    """Every interior face's traction enters its two cells with opposite
    signs and z is periodic, so a velocity field that vanishes near the
    walls feels no net viscous force, whatever the viscosities."""
    g = Grid(12, 11, 10, h=0.25e-3)
    a = sphere_alpha(g, [[6.1 * g.h, 5.4 * g.h, 4.7 * g.h]], 3.3 * g.h)
    a = np.clip(a + 0.2 * np.random.default_rng(5).uniform(-1, 1, a.shape) * (a < 1), 0, 1)
    ph = Phys()  # water and air: mu jumps by 55
    rng = np.random.default_rng(6)
    q = []
    for _ in range(3):
        f = rng.normal(size=g.shapes()[0])
        f[:, :2, :] = f[:, -2:, :] = 0.0
        f[:, :, :2] = f[:, :, -2:] = 0.0
        q.append(f)
    V = viscous(g, ph, a, q)
    for Vc in V:
        assert np.abs(Vc).max() > 0
        assert abs(np.sum(Vc)) <= 1e-12 * np.sum(np.abs(Vc))


def test_two_fluid_shear_layer_with_uniform_traction_is_in_equilibrium():
    """w(x) across a liquid/gas layer (mu_l / mu_g = 55, one cell partly
    filled) built so that the discrete shear traction is the same tau on
    every x face, the wall face included: the viscous force vanishes in
    every cell whose faces all carry that traction."""
    g = Grid(10, 6, 5, h=0.25e-3)
    ph = Phys()
    ax = np.array([1, 1, 1, 1, 0.37, 0, 0, 0, 0, 0], dtype=np.float64)
    a = np.broadcast_to(ax, g.shapes()[0]).copy()
    mu = ax * ph.mu_l + (1 - ax) * ph.mu_g
    tau = 2.5e-3
    w = np.zeros(g.nx)
    w[0] = tau * g.h / (2 * mu[0])  # wall face: ghost -w[0], face viscosity mu[0]
    for i in range(g.nx - 1):
        w[i + 1] = w[i] + tau * g.h / (0.5 * (mu[i] + mu[i + 1]))
    wc = np.broadcast_to(w, g.shapes()[0]).copy()
    z = np.zeros(g.shapes()[0])
    _, _, Vz = viscous(g, ph, a, [z, z, wc])
    inner = Vz[:, 1:-1, :-1]  # not the y walls (w does not vanish there), not the far x wall
    ref = tau / g.h  # the size of one face's contribution
    assert np.max(np.abs(inner)) <= 1e-9 * ref
    # the far wall feels the traction difference
    assert np.min(np.abs(Vz[:, 1:-1, -1])) > 0.1 * ref
