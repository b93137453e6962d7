"""Pins of the oracle's geometric VOF advection (Eq. 3; split geometric
fluxes, Section 2.1): exact donor-slab volumes, exact translation at unit
Courant number, and conservation of liquid volume to round-off."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2104_01636_b300.inputs import Grid, curl_noise, sphere_alpha
from test_oracle_geometry import exact_halfspace_volume


def _sphere_grid(n=16, nz=None, R=4.0, per=False, off=(0.3, -0.2, 0.1)):
    nz = nz or n
    g = Grid(n, n, nz, per_x=int(per), per_y=int(per))
    c = np.array([[(n / 2 + off[0]) * g.h, (n / 2 + off[1]) * g.h, (nz / 2 + off[2]) * g.h]])
    return g, sphere_alpha(g, c, R * g.h)


@pytest.mark.parametrize("U", [+1.0, -1.0])
def test_single_face_flux_is_exact_slab_volume(U):
    g, a = _sphere_grid(10, R=2.6)
    cs, us, vs, ws = g.shapes()
    # pick an x-face whose donor is an interface cell
    k, j = 5, 4
    i_face = None
    for i in range(1, g.nx):
        donor = i - 1 if U > 0 else i
        if 0.05 < a[k, j, donor] < 0.95:
            i_face = i
            break
    assert i_face is not None
    donor = i_face - 1 if U > 0 else i_face
    u = np.zeros(us)
    u[k, j, i_face] = U
    c = 0.3
    dt = c * g.h / abs(U)
    a_new, rep = oracle.advect(g, a, u, np.zeros(vs), np.zeros(ws), dt, 0)
    cd = 1.0 if a[k, j, donor] > 0.5 else 0.0
    # the donor loses the flux; its divergence term is +c in both directions
    # (U dt/h on its plus face, or -U dt/h on its minus face)
    div_term = cd * c
    F = a[k, j, donor] - a_new[k, j, donor] + div_term
    n = oracle.normal(g, a, donor, j, k)
    d = oracle.plane_constant(n, a[k, j, donor])
    fc = Fraction(c)
    lo = (1 - fc, 0, 0) if U > 0 else (0, 0, 0)
    hi = (1, 1, 1) if U > 0 else (fc, 1, 1)
    exact = exact_halfspace_volume([Fraction(x) for x in n], Fraction(d), lo, hi)
    assert F == pytest.approx(float(exact), abs=2e-15)
    assert 0 < F <= c
    # every other cell except donor/acceptor is unchanged
    mask = np.ones(cs, bool)
    mask[k, j, i_face - 1:i_face + 1] = False
    assert np.array_equal(a_new[mask], a[mask])


def test_unit_courant_translation_is_exact():
    g, a0 = _sphere_grid(12, nz=16, R=4.0)
    cs, us, vs, ws = g.shapes()
    w = np.full(ws, 0.05)
    dt = g.h / 0.05
    a, _ = oracle.advect(g, a0, np.zeros(us), np.zeros(vs), w, dt, 0)
    assert np.max(np.abs(a - np.roll(a0, 1, axis=0))) < 1e-13
    for s in range(1, g.nz):
        a, _ = oracle.advect(g, a, np.zeros(us), np.zeros(vs), w, dt, s)
    assert np.max(np.abs(a - a0)) < 1e-12


def test_unit_courant_translation_periodic_x():
    g, a0 = _sphere_grid(12, nz=8, R=3.0, per=True)
    cs, us, vs, ws = g.shapes()
    u = np.full(us, -0.2)
    dt = g.h / 0.2
    a, _ = oracle.advect(g, a0, u, np.zeros(vs), np.zeros(ws), dt, 1)
    assert np.max(np.abs(a - np.roll(a0, -1, axis=2))) < 1e-13


def test_volume_conserved_for_solenoidal_field():
    g, a = _sphere_grid(16, nz=24, R=5.0)
    u, v, w = curl_noise(g, 0.1, seed=11, kmax=3)
    w = w + 0.05
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    dt = 0.45 * g.h / umax
    vol0 = a.sum()
    for s in range(8):
        a, rep = oracle.advect(g, a, u, v, w, dt, s)
        assert rep["vol_after"] == pytest.approx(rep["vol_before"] + rep["vol_clipped"] * 0, rel=1e-13)
        assert a.min() >= 0.0 and a.max() <= 1.0
        assert abs(rep["vol_clipped"]) < 1e-10 * rep["vol_before"]
    assert abs(a.sum() - vol0) < 1e-13 * vol0


def test_wall_face_values_are_ignored():
    g, a = _sphere_grid(10, R=3.0)
    cs, us, vs, ws = g.shapes()
    u, v, w = curl_noise(g, 0.1, seed=12, kmax=2)
    dt = 0.3 * g.h / max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    ref, _ = oracle.advect(g, a, u, v, w, dt, 0)
    u2, v2 = u.copy(), v.copy()
    u2[:, :, 0] = 5.0
    u2[:, :, -1] = -3.0
    v2[:, 0, :] = 2.0
    got, _ = oracle.advect(g, a, u2, v2, w, dt, 0)
    assert np.array_equal(ref, got)


def test_diagonal_translation_returns_near_start():
    """All-periodic box, uniform (U,U,U) at Courant 1/4: after one period
    the sphere returns with a small shape error and exactly its volume."""
    g, a0 = _sphere_grid(16, R=4.0, per=True)
    cs, us, vs, ws = g.shapes()
    U = 0.1
    dt = 0.25 * g.h / U
    a = a0
    for s in range(64):
        a, rep = oracle.advect(g, a, np.full(us, U), np.full(vs, U), np.full(ws, U), dt, s)
    assert abs(a.sum() - a0.sum()) < 1e-12 * a0.sum()
    l1 = np.abs(a - a0).sum() / (1.0 - a0).sum()
    assert l1 < 0.25
