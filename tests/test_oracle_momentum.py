"""Pins of the oracle's momentum predictor (Eq. 2; steps 8-10): the viscous
operator's steady duct solution against the textbook series, the discrete
consistency of momentum transport with the VOF mass fluxes (uniform flow is
kept exactly across density jumps; upwind transport of a one-directional flow
is a convex combination),
the skew-symmetry and conservation of central transport, and the body force
with the hydrostatic part removed (Section 4)."""
import numpy as np
import pytest

import oracle
from paper_2104_01636_b300.inputs import (GRAV, Grid, Phys, curl_noise, face_to_cell,
                                          laminar_duct_profile, sphere_alpha)


def _zeros(g):
    cs, us, vs, ws = g.shapes()
    return np.zeros(cs), np.zeros(us), np.zeros(vs), np.zeros(ws)


def _laminar_error(n):
    """Steady state of the predictor (alpha = 1, no face flow) for a
    z-independent cell w driven by G, against the exact series."""
    g = Grid(n, n, 4)
    G = 3.0
    ph = Phys(dpdz=G, rho0=1000.0)
    c0, u0, v0, w0 = _zeros(g)
    a = np.ones(g.shapes()[0])
    dt = 1.0
    flux = (u0, v0, w0)

    def Vop(wc):  # dt (V(w) + G) = rho w_hat - rho w
        return 1000.0 * (oracle.predict(g, ph, a, a, c0, c0, wc, u0, v0, w0, *flux, dt)[2] - wc)

    base = Vop(np.zeros_like(c0))[0].ravel()
    A = np.zeros((n * n, n * n))
    for col in range(n * n):
        e = np.zeros_like(c0)
        e[:, col // n, col % n] = 1.0
        A[:, col] = Vop(e)[0].ravel() - base
    wd = np.linalg.solve(A, -base)
    x = (np.arange(n) + 0.5) * g.h
    exact = laminar_duct_profile(x[None, :], x[:, None], n * g.h, G, ph.mu_l).ravel()
    return np.max(np.abs(wd - exact)) / np.max(exact)


def test_viscous_operator_laminar_duct_second_order():
    e1, e2 = _laminar_error(12), _laminar_error(24)
    assert e1 < 0.02
    assert e2 < e1 / 3.0  # second order in h


def test_body_force_with_hydrostatic_removal():
    g = Grid(6, 5, 4)
    c0, u0, v0, w0 = _zeros(g)
    ph = Phys(g_z=-GRAV, rho0=990.0, dpdz=2.5)
    a = np.ones(g.shapes()[0])
    dt = 1e-4
    uh, vh, wh = oracle.predict(g, ph, a, a, c0, c0, c0, u0, v0, w0, u0, v0, w0, dt)
    assert np.all(uh == 0) and np.all(vh == 0)
    assert np.allclose(wh, dt * ((1000.0 - 990.0) * -GRAV + 2.5) / 1000.0, rtol=1e-14, atol=0)


def _bubbles(g, seed=3):
    rng = np.random.default_rng(seed)
    c = np.array([[rng.uniform(3, g.nx - 3) * g.h, rng.uniform(3, g.ny - 3) * g.h,
                   rng.uniform(0, g.nz) * g.h] for _ in range(2)])
    return sphere_alpha(g, c, 2.4 * g.h)


@pytest.mark.parametrize("scheme", [0, 1])
def test_uniform_flow_is_kept_exactly_across_density_jumps(scheme):
    """Mass-momentum consistency: a uniform velocity carried through gas
    bubbles at density ratio 833 stays uniform to round-off, because the
    momentum moves with the same mass fluxes that move alpha."""
    g = Grid(10, 9, 16)
    a0 = _bubbles(g)
    c0, u0, v0, w0 = _zeros(g)
    W = 0.3
    w = np.full(g.shapes()[3], W)
    dt = 0.4 * g.h / W
    ph = Phys(mu_l=0.0, mu_g=0.0, conv_scheme=scheme)
    a1, fl, _ = oracle.advect(g, a0, u0, v0, w, dt, 0, fluxes=True)
    assert np.max(np.abs(a1 - a0)) > 0.05  # the bubbles did move
    uh, vh, wh = oracle.predict(g, ph, a0, a1, c0, c0, np.full_like(c0, W), u0, v0, w, *fl, dt)
    assert np.max(np.abs(uh)) == 0 and np.max(np.abs(vh)) == 0
    assert np.max(np.abs(wh - W)) < 1e-13 * W


def test_upwind_transport_is_bounded_for_one_directional_flow():
    """When mass moves in one direction only (w(x, y), uniform in z), the
    upwind update is a convex combination of the old cell values (the donor
    slab never holds more mass than its cell), so it creates no new extrema.
    With flow in several directions the split sweeps break this bound at
    second order, so the general case is not pinned."""
    g = Grid(12, 10, 14)
    a0 = _bubbles(g, 5)
    c0, u0, v0, _ = _zeros(g)
    rng = np.random.default_rng(8)
    w = np.broadcast_to(rng.uniform(-0.2, 0.2, (g.ny, g.nx)), g.shapes()[3]).copy()
    dt = 0.9 * g.h / np.abs(w).max()
    a1, fl, _ = oracle.advect(g, a0, u0, v0, w, dt, 1, fluxes=True)
    q = [rng.uniform(-1, 1, g.shapes()[0]) for _ in range(3)]
    ph = Phys(mu_l=0.0, mu_g=0.0, conv_scheme=1)
    out = oracle.predict(g, ph, a0, a1, *q, u0, v0, w, *fl, dt)
    for qh, q0 in zip(out, q):
        assert qh.max() <= q0.max() + 1e-12 and qh.min() >= q0.min() - 1e-12


def test_central_transport_is_skew_symmetric_and_conservative():
    g = Grid(10, 8, 12)
    u, v, w = curl_noise(g, 0.2, seed=21, kmax=3)
    a = np.ones(g.shapes()[0])
    dt = 0.3 * g.h / max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    a1, fl, _ = oracle.advect(g, a, u, v, w, dt, 0, fluxes=True)
    assert np.max(np.abs(a1 - 1.0)) < 1e-14
    rng = np.random.default_rng(9)
    q = [rng.normal(size=g.shapes()[0]) for _ in range(3)]
    ph = Phys(mu_l=0.0, mu_g=0.0, conv_scheme=0)
    out = oracle.predict(g, ph, a, a1, *q, u, v, w, *fl, dt)
    for qh, q0 in zip(out, q):
        C = 1000.0 * (q0 - qh)  # rho^n q - rho^{n+1} q_hat with rho = rho_l
        assert abs(np.sum(q0 * C)) < 1e-12 * np.sum(np.abs(q0 * C))
        assert abs(np.sum(C)) < 1e-12 * np.sum(np.abs(C))


@pytest.mark.parametrize("scheme", [0, 1])
def test_streamwise_momentum_conserved_with_bubbles(scheme):
    g = Grid(9, 8, 10)
    a0 = _bubbles(g, 11)
    u, v, w = curl_noise(g, 0.2, seed=22, kmax=3)
    w = w + 0.1
    dt = 0.3 * g.h / max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    a1, fl, _ = oracle.advect(g, a0, u, v, w, dt, 0, fluxes=True)
    uc, vc, wc = face_to_cell(u, v, w)
    ph = Phys(mu_l=0.0, mu_g=0.0, conv_scheme=scheme)
    _, _, wh = oracle.predict(g, ph, a0, a1, uc, vc, wc, u, v, w, *fl, dt)
    rho0 = a0 * 1000.0 + (1 - a0) * 1.2
    rho1 = a1 * 1000.0 + (1 - a1) * 1.2
    m0, m1 = np.sum(rho0 * wc), np.sum(rho1 * wh)
    assert abs(m1 - m0) < 1e-12 * np.sum(np.abs(rho0 * wc))


def test_cell_to_face_is_linear_average():
    g = Grid(5, 4, 6)
    rng = np.random.default_rng(3)
    uc, vc, wc = (rng.normal(size=g.shapes()[0]) for _ in range(3))
    u, v, w = oracle.cell_to_face(g, uc, vc, wc)
    assert u[2, 1, 3] == pytest.approx(0.5 * (uc[2, 1, 2] + uc[2, 1, 3]), rel=1e-15)
    assert v[3, 2, 4] == pytest.approx(0.5 * (vc[3, 1, 4] + vc[3, 2, 4]), rel=1e-15)
    assert w[0, 1, 1] == pytest.approx(0.5 * (wc[-1, 1, 1] + wc[0, 1, 1]), rel=1e-15)
    assert np.all(u[:, :, 0] == 0) and np.all(u[:, :, -1] == 0)
    assert np.all(v[:, 0, :] == 0) and np.all(v[:, -1, :] == 0)
