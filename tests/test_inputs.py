"""Checks of the seeded input generator against the paper's printed
parameters and against the mathematical properties it promises."""
import json
import math
import os

import numpy as np
import pytest

from paper_2104_01636_b300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")))
V = {k: v["value"] for k, v in GOLDEN["values"].items()}


def test_paper_parameters_are_consistent():
    assert I.RHO_L == V["rho_l"] and I.RHO_G == V["rho_g"] and I.MU_L == V["mu_l"]
    assert I.SIGMA == V["sigma"]
    assert I.H_PAPER == pytest.approx(V["duct"][0] / V["grid"][0], rel=1e-15)
    assert V["rho_l"] / V["rho_g"] == pytest.approx(V["density_ratio"], abs=0.5)
    d = V["d_bubble"]
    bo = V["rho_l"] * I.GRAV * d * d / V["sigma"]
    mo = I.GRAV * V["mu_l"] ** 4 / (V["rho_l"] * V["sigma"] ** 3)
    assert bo == pytest.approx(V["bond"], abs=0.01)
    assert mo == pytest.approx(V["morton"], rel=0.02)
    phi = V["n_bubbles"] * math.pi / 6 * d ** 3 / np.prod(V["duct"])
    assert phi == pytest.approx(V["void_fraction"], abs=2e-4)
    assert np.prod(V["array"]) == V["n_bubbles"]
    u_tau = V["re_tau"] * V["mu_l"] / (V["rho_l"] * V["duct"][0])
    assert u_tau * I.H_PAPER / (V["mu_l"] / V["rho_l"]) == pytest.approx(V["dx_plus"], rel=1e-12)


def test_sphere_volume_and_bounds():
    g = I.Grid(40, 40, 40)
    R = 9.3 * g.h
    a = I.sphere_alpha(g, np.array([[20.2 * g.h, 19.6 * g.h, 20.9 * g.h]]), R)
    gas = (1 - a).sum() * g.h ** 3
    assert gas == pytest.approx(4 / 3 * math.pi * R ** 3, rel=2e-4)
    assert a.min() >= 0 and a.max() <= 1
    # periodic wrap in z
    a2 = I.sphere_alpha(g, np.array([[20.2 * g.h, 19.6 * g.h, 0.4 * g.h]]), R)
    assert (1 - a2).sum() * g.h ** 3 == pytest.approx(gas, rel=1e-3)


def test_sphere_placement_constraints():
    g = I.Grid(64, 64, 128)
    d = 12 * g.h
    c = I.place_spheres(g, 8, d, seed=2104)
    assert c.shape == (8, 3)
    L = g.nz * g.h
    for i in range(8):
        assert d / 2 + g.h <= c[i, 0] <= g.nx * g.h - d / 2 - g.h
        for j in range(i):
            dz = abs(c[i, 2] - c[j, 2])
            dz = min(dz, L - dz)
            assert math.hypot(math.hypot(c[i, 0] - c[j, 0], c[i, 1] - c[j, 1]), dz) >= d + 2 * g.h
    assert np.array_equal(c, I.place_spheres(g, 8, d, seed=2104))  # seeded


def test_curl_noise_is_solenoidal_with_zero_wall_flux():
    g = I.Grid(12, 10, 16)
    u, v, w = I.curl_noise(g, 0.05, seed=3)
    assert np.all(u[:, :, 0] == 0) and np.all(u[:, :, -1] == 0)
    assert np.all(v[:, 0, :] == 0) and np.all(v[:, -1, :] == 0)
    tot = np.concatenate([u.ravel(), v.ravel(), w.ravel()])
    assert math.sqrt(np.mean(tot ** 2)) == pytest.approx(0.05, rel=1e-12)
    assert np.max(np.abs(I.divergence(g, u, v, w))) < 1e-12 * 0.05 / g.h


def test_laminar_series_solves_the_duct_problem():
    """The series against an independent sparse finite-difference solve of
    mu (w_xx + w_yy) = -G with w = 0 on the walls (second-order, n = 160)."""
    import scipy.sparse as sps
    import scipy.sparse.linalg as spl
    W, G, mu = 0.016, 4.0, 1e-3
    n = 160
    hx = W / n
    x = (np.arange(n) + 0.5) * hx
    w = I.laminar_duct_profile(x[None, :], x[:, None], W, G, mu)
    # cell-centred Laplacian with Dirichlet walls (ghost = -interior)
    main = -2 * np.ones(n)
    main[0] = main[-1] = -3
    T = sps.diags([np.ones(n - 1), main, np.ones(n - 1)], [-1, 0, 1]) / hx ** 2
    L = sps.kron(sps.eye(n), T) + sps.kron(T, sps.eye(n))
    wfd = spl.spsolve(L.tocsc(), -G / mu * np.ones(n * n)).reshape(n, n)
    assert np.max(np.abs(w - wfd)) < 2e-4 * w.max()
    edge = I.laminar_duct_profile(np.array([0.0, W]), np.array([W / 3, W / 3]), W, G, mu)
    assert np.max(np.abs(edge)) < 1e-9 * w.max()
    # the known square-duct ratio of mean to centre velocity (about 0.477)
    assert w.mean() / w.max() == pytest.approx(0.4770, abs=2e-3)


def test_workloads_build_small():
    c = I.static_bubble()
    assert c.grid.ncells == 32 ** 3 and c.dt > 0
    s = I.rising_swarm(32, 32, 48, nbub=3, seed=1, steps=1)
    assert np.max(np.abs(I.divergence(s.grid, s.u, s.v, s.w))) < 1e-9
    assert 0 < s.phys.rho0 < I.RHO_L
