"""Pins of the oracle's momentum predictor (Eq. 2; steps 8-10): the viscous
operator's steady duct solution against the textbook series, the discrete
skew-symmetry and conservation of the central convective term, and the body
force with the hydrostatic part removed (Section 4)."""
import numpy as np
import pytest

import oracle
from paper_2104_01636_b300.inputs import (GRAV, Grid, Phys, curl_noise, laminar_duct_profile,
                                          sphere_alpha)


def _laminar_error(n):
    """Discrete steady state of the predictor (alpha = 1, u = v = 0) for a
    z-independent w driven by G, against the exact series solution."""
    g = Grid(n, n, 2)
    G = 3.0
    ph = Phys(dpdz=G, rho0=1000.0)
    cs, us, vs, ws = g.shapes()
    a = np.ones(cs)
    dt = 1.0
    # the predictor is affine in w here: M(w) = rho w + dt (V(w) + G)
    base = oracle.momentum(g, ph, a, np.zeros(us), np.zeros(vs), np.zeros(ws), dt)[2][0].ravel()
    A = np.zeros((n * n, n * n))
    for col in range(n * n):
        w = np.zeros(ws)
        w[:, col // n, col % n] = 1.0
        Mw = oracle.momentum(g, ph, a, np.zeros(us), np.zeros(vs), w, dt)[2][0].ravel()
        A[:, col] = Mw - base - 1000.0 * w[0].ravel()  # = dt * V(e_col)
    wd = np.linalg.solve(A, -base)  # V(w) + G = 0
    x = (np.arange(n) + 0.5) * g.h
    exact = laminar_duct_profile(x[None, :], x[:, None], n * g.h, G, ph.mu_l).ravel()
    return np.max(np.abs(wd - exact)) / np.max(exact)


def test_viscous_operator_laminar_duct_second_order():
    e1, e2 = _laminar_error(12), _laminar_error(24)
    assert e1 < 0.02
    assert e2 < e1 / 3.0  # second order in h


def test_body_force_with_hydrostatic_removal():
    g = Grid(6, 5, 4)
    cs, us, vs, ws = g.shapes()
    ph = Phys(g_z=-GRAV, rho0=990.0, dpdz=2.5)
    a = np.ones(cs)
    dt = 1e-4
    Mu, Mv, Mw = oracle.momentum(g, ph, a, np.zeros(us), np.zeros(vs), np.zeros(ws), dt)
    assert np.all(Mu == 0) and np.all(Mv == 0)
    assert np.allclose(Mw, dt * ((1000.0 - 990.0) * -GRAV + 2.5), rtol=1e-14, atol=0)


def _convection(g, a, u, v, w, scheme):
    ph = Phys(mu_l=0.0, mu_g=0.0, conv_scheme=scheme)
    dt = 1.0
    rho = a * ph.rho_l + (1 - a) * ph.rho_g
    Mu, Mv, Mw = oracle.momentum(g, ph, a, u, v, w, dt)
    rfx = 0.5 * (rho[:, :, 1:] + rho[:, :, :-1])
    rfy = 0.5 * (rho[:, 1:, :] + rho[:, :-1, :])
    rfz = 0.5 * (rho + np.roll(rho, 1, axis=0))
    Cu = np.zeros_like(u)
    Cv = np.zeros_like(v)
    Cu[:, :, 1:-1] = rfx * u[:, :, 1:-1] - Mu[:, :, 1:-1]
    Cv[:, 1:-1, :] = rfy * v[:, 1:-1, :] - Mv[:, 1:-1, :]
    Cw = rfz * w - Mw
    return Cu, Cv, Cw


def test_central_convection_is_skew_symmetric():
    g = Grid(10, 8, 12)
    u, v, w = curl_noise(g, 0.2, seed=21, kmax=3)
    a = np.ones(g.shapes()[0])
    Cu, Cv, Cw = _convection(g, a, u, v, w, 0)
    e = np.sum(u * Cu) + np.sum(v * Cv) + np.sum(w * Cw)
    scale = np.sum(np.abs(u * Cu)) + np.sum(np.abs(v * Cv)) + np.sum(np.abs(w * Cw))
    assert abs(e) < 1e-13 * scale
    # the first-order upwind form dissipates energy instead
    Uu, Uv, Uw = _convection(g, a, u, v, w, 1)
    assert np.sum(u * Uu) + np.sum(v * Uv) + np.sum(w * Uw) > 1e-6 * scale


@pytest.mark.parametrize("scheme", [0, 1])
def test_convection_conserves_streamwise_momentum(scheme):
    """Periodic in z and no mass flux through the walls: the convective
    fluxes of w-momentum telescope to zero, with variable density too."""
    g = Grid(9, 8, 10)
    u, v, w = curl_noise(g, 0.2, seed=22, kmax=3)
    a = sphere_alpha(g, np.array([[4.3 * g.h, 4.1 * g.h, 5.2 * g.h]]), 2.5 * g.h)
    _, _, Cw = _convection(g, a, u, v, w + 0.1, scheme)
    assert abs(Cw.sum()) < 1e-13 * np.abs(Cw).sum()
