"""Pins of the oracle's variable-coefficient pressure operator and solver
(Eq. 7 and steps 6/11: div(grad p / rho) with beta = 1/rho on faces)."""
import math

import numpy as np
import pytest

import oracle
from paper_2104_01636_b300.inputs import Grid, Phys, sphere_alpha


def _cos_mode(g, px=1, py=1, pz=1):
    h = g.h
    x = (np.arange(g.nx) + 0.5) * h
    y = (np.arange(g.ny) + 0.5) * h
    z = (np.arange(g.nz) + 0.5) * h
    W, Wy, L = g.nx * h, g.ny * h, g.nz * h
    return (np.cos(pz * 2 * np.pi * z / L)[:, None, None] * np.cos(py * np.pi * y / Wy)[None, :, None]
            * np.cos(px * np.pi * x / W)[None, None, :])


def _const_beta(g, c=1.0):
    _, us, vs, ws = g.shapes()
    bx, by, bz = np.full(us, c), np.full(vs, c), np.full(ws, c)
    bx[:, :, 0] = bx[:, :, -1] = 0.0
    by[:, 0, :] = by[:, -1, :] = 0.0
    return bx, by, bz


@pytest.mark.parametrize("dims", [(8, 8, 8), (12, 10, 16), (5, 7, 6)])
def test_operator_discrete_eigenfunction(dims):
    """cos(pi x/W) cos(pi y/W) cos(2 pi z/L) sampled at cell centres is an
    exact eigenvector of the wall-Neumann / z-periodic 7-point operator,
    with eigenvalue sum over axes of 2(1 - cos(theta))/h^2."""
    g = Grid(*dims, h=0.37)
    c = 2.5
    bx, by, bz = _const_beta(g, c)
    for px, py, pz in [(1, 1, 1), (2, 0, 1), (0, 3, 2)]:
        P = _cos_mode(g, px, py, pz)
        lam = c * (2 * (1 - math.cos(px * math.pi / g.nx)) + 2 * (1 - math.cos(py * math.pi / g.ny)) +
                   2 * (1 - math.cos(pz * 2 * math.pi / g.nz))) / g.h ** 2
        AP = oracle.apply_A(g, bx, by, bz, P)
        assert np.max(np.abs(AP - lam * P)) < 1e-12 * lam * np.max(np.abs(P))


def _random_beta(g, seed):
    rng = np.random.default_rng(seed)
    _, us, vs, ws = g.shapes()
    bx, by, bz = rng.uniform(0.001, 1.0, us), rng.uniform(0.001, 1.0, vs), rng.uniform(0.001, 1.0, ws)
    bx[:, :, 0] = bx[:, :, -1] = 0.0
    by[:, 0, :] = by[:, -1, :] = 0.0
    return bx, by, bz


def test_operator_symmetric_psd_constant_nullspace():
    g = Grid(7, 6, 9, h=0.5)
    bx, by, bz = _random_beta(g, 4)
    rng = np.random.default_rng(5)
    x, y = rng.normal(size=(2,) + g.shapes()[0])
    Ax, Ay = oracle.apply_A(g, bx, by, bz, x), oracle.apply_A(g, bx, by, bz, y)
    assert np.sum(x * Ay) == pytest.approx(np.sum(Ax * y), rel=1e-13)
    assert np.sum(x * Ax) > 0
    one = np.ones(g.shapes()[0]) * 3.7
    assert np.max(np.abs(oracle.apply_A(g, bx, by, bz, one))) == 0.0
    # the quadratic form is the face-difference energy
    h2 = g.h ** 2
    e = (np.sum(bx[:, :, 1:-1] * (x[:, :, 1:] - x[:, :, :-1]) ** 2) +
         np.sum(by[:, 1:-1, :] * (x[:, 1:, :] - x[:, :-1, :]) ** 2) +
         np.sum(bz * (x - np.roll(x, 1, axis=0)) ** 2)) / h2
    assert np.sum(x * Ax) == pytest.approx(e, rel=1e-13)


def test_beta_is_inverse_linear_face_density():
    g = Grid(6, 5, 4)
    ph = Phys()
    rng = np.random.default_rng(6)
    a = rng.uniform(0, 1, g.shapes()[0])
    bx, by, bz = oracle.beta(g, ph, a)
    rho = a * ph.rho_l + (1 - a) * ph.rho_g
    assert bx[2, 3, 4] == pytest.approx(2.0 / (rho[2, 3, 3] + rho[2, 3, 4]), rel=1e-15)
    assert by[1, 2, 0] == pytest.approx(2.0 / (rho[1, 1, 0] + rho[1, 2, 0]), rel=1e-15)
    assert bz[0, 1, 2] == pytest.approx(2.0 / (rho[-1, 1, 2] + rho[0, 1, 2]), rel=1e-15)
    assert np.all(bx[:, :, 0] == 0) and np.all(bx[:, :, -1] == 0)
    assert np.all(by[:, 0, :] == 0) and np.all(by[:, -1, :] == 0)


def test_solve_eigenmode_exact():
    g = Grid(12, 12, 16)
    bx, by, bz = _const_beta(g, 1e-3)
    P = _cos_mode(g)
    lam = 1e-3 * (4 * (1 - math.cos(math.pi / 12)) + 2 * (1 - math.cos(2 * math.pi / 16))) / g.h ** 2
    sol, rep, st = oracle.solve(g, bx, by, bz, lam * P, rtol=1e-13)
    assert st == 0 and rep["res"] <= 1e-13
    assert np.max(np.abs(sol - P)) < 1e-10


def test_solve_manufactured_high_density_ratio():
    """b := A P* with beta from a gas sphere at rho_l/rho_g = 833; the solve
    must return P* (mean-free) to the accuracy its residual allows."""
    g = Grid(16, 16, 24)
    a = sphere_alpha(g, np.array([[8.3 * g.h, 7.6 * g.h, 12.2 * g.h]]), 5 * g.h)
    bx, by, bz = oracle.beta(g, Phys(), a)
    P = _cos_mode(g) + 0.3 * _cos_mode(g, 2, 1, 0)
    P -= P.mean()
    b = oracle.apply_A(g, bx, by, bz, P)
    sol, rep, st = oracle.solve(g, bx, by, bz, b, rtol=1e-12)
    assert st == 0
    assert abs(rep["b_mean"]) < 1e-12 * np.max(np.abs(b))
    assert np.abs(sol.mean()) < 1e-14
    assert np.linalg.norm(sol - P) / np.linalg.norm(P) < 1e-8
    # a non-mean-free right side: the solver removes (and reports) the mean
    sol2, rep2, st2 = oracle.solve(g, bx, by, bz, b + 5.0, rtol=1e-12)
    assert st2 == 0 and rep2["b_mean"] == pytest.approx(5.0, rel=1e-12)
    assert np.linalg.norm(sol2 - P) / np.linalg.norm(P) < 1e-8


def test_solve_zero_rhs_and_nonconvergence_flag():
    g = Grid(6, 6, 6)
    bx, by, bz = _const_beta(g)
    sol, rep, st = oracle.solve(g, bx, by, bz, np.zeros(g.shapes()[0]), rtol=1e-12)
    assert st == 0 and np.all(sol == 0)
    b = np.random.default_rng(7).normal(size=g.shapes()[0])
    _, rep, st = oracle.solve(g, bx, by, bz, b, rtol=1e-14, max_iter=2)
    assert st == 1 and rep["iters"] == 2
