"""Pins of the statistics oracle: closed forms of z-averages, Reynolds
stresses of a known oscillation, liquid-only weighting, quadrant folding."""
import numpy as np

from oracle import stats as S
from paper_2104_01636_b300 import fold_quadrants


def test_uniform_fields():
    nz, ny, nx = 8, 3, 4
    a = np.full((nz, ny, nx), 0.75)
    u, v, w = (np.full((nz, ny, nx), c) for c in (0.5, -0.25, 2.0))
    m = S.means(S.column_sums(a, u, v, w), 1, nz)
    assert np.allclose(m["phi"], 0.25) and np.allclose(m["w"], 2.0)
    assert np.allclose(m["uv"], -0.125) and np.allclose(m["rs_ww"], 0.0, atol=1e-15)
    assert np.allclose(m["l_u"], 0.5)


def test_oscillation_mean_and_stress_closed_form():
    """w = B + A sin(2 pi m k / nz): over whole periods the z-mean is B and
    the stress <w'w'> is A^2/2 exactly (sum of sin^2 = nz/2 for 0 < m < nz/2)."""
    nz, ny, nx, A, B, m = 64, 2, 2, 0.3, 1.7, 5
    k = np.arange(nz)[:, None, None]
    w = B + A * np.sin(2 * np.pi * m * k / nz) * np.ones((1, ny, nx))
    z = np.zeros((nz, ny, nx))
    res = S.means(S.column_sums(np.ones_like(w), z, z, w), 1, nz)
    assert np.allclose(res["w"], B, rtol=0, atol=1e-14)
    assert np.allclose(res["rs_ww"], A * A / 2, rtol=1e-12)
    assert np.allclose(res["rs_uw"], 0.0, atol=1e-15)


def test_liquid_weighting_selects_liquid_cells():
    nz, ny, nx = 10, 1, 1
    a = np.zeros((nz, ny, nx))
    a[:4] = 1.0  # liquid in the first four planes
    u = np.arange(nz, dtype=float)[:, None, None] * np.ones((1, ny, nx))
    z = np.zeros_like(u)
    res = S.means(S.column_sums(a, u, z, z), 1, nz)
    assert res["l_u"][0, 0] == np.mean(np.arange(4))
    assert res["u"][0, 0] == np.mean(np.arange(nz))
    assert res["phi"][0, 0] == 0.6


def test_fold_quadrants_parities():
    ny = nx = 6
    y, x = np.meshgrid(np.arange(ny) - 2.5, np.arange(nx) - 2.5, indexing="ij")
    even = x * x + y * y
    odd_x = x * (1 + y * y)
    assert np.allclose(fold_quadrants(even), even)
    assert np.allclose(fold_quadrants(odd_x, parity_x=-1), odd_x)
    assert np.allclose(fold_quadrants(odd_x), 0.0)
