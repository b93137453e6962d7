"""Pins of the oracle's face curvature in the sharp surface force (Eq. 6;
steps 5-7): the face value is the mean of the valid height-function values
of its two cells, else the one valid value, else the mean over the valid
cells of the 2 x 3 x 3 block around the face, else 0 (each use of the block
counted as a fallback).

* Where both cells are valid, the face value is checked against the
  symbolic curvature of a quadratic height surface at the two column
  centres (the height function is exact there), so a face value taken from
  one cell only, or from the wrong pair, fails.
* The fallbacks fire around the caps of a finite gas cylinder and on a gas
  pocket of whole cells (no valid cell near it): every face
  force is recovered as kappa_f = s_f h / (sigma (G_R - G_L)) and checked,
  face by face, against a brute-force enumeration of the branches over the
  cells' curvatures and validity flags, with every branch required to fire;
  the fallback count must equal the number of faces that used the block.
  Independently of the branches, the side faces carry 1/R to within the
  height function's accuracy and the flat caps carry exactly 0.
"""
import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2104_01636_b300.inputs import Grid, Phys

SIGMA = 0.5


def face_kappas(g, alpha):
    """(direction, left cell (k, j, i), kappa_f) for every face whose gas
    indicator jumps, read off the oracle's face forces."""
    ph = Phys(sigma=SIGMA, kappa_mode=0)
    kap, sx, sy, sz, rep = oracle.ssf(g, ph, alpha)
    G = (alpha < 0.5).astype(np.float64)
    out = []
    nz, ny, nx = alpha.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if i + 1 < nx and G[k, j, i + 1] != G[k, j, i]:
                    out.append((0, (k, j, i), sx[k, j, i + 1] * g.h /
                                (SIGMA * (G[k, j, i + 1] - G[k, j, i]))))
                if j + 1 < ny and G[k, j + 1, i] != G[k, j, i]:
                    out.append((1, (k, j, i), sy[k, j + 1, i] * g.h /
                                (SIGMA * (G[k, j + 1, i] - G[k, j, i]))))
                kn = (k + 1) % nz
                if G[kn, j, i] != G[k, j, i]:
                    out.append((2, (k, j, i), sz[kn, j, i] * g.h /
                                (SIGMA * (G[kn, j, i] - G[k, j, i]))))
    return kap, out, rep


def right_of(d, c, shape):
    k, j, i = c
    return ((k + 1) % shape[0], j, i) if d == 2 else ((k, j + 1, i) if d == 1 else (k, j, i + 1))


# --- both cells valid: against the symbolic curvature of a quadric ----------------
def test_face_value_with_two_valid_cells_is_their_mean_curvature():
    Xs, Ys = sp.symbols("x y")
    f = 8.3 + 0.17 * Xs - 0.11 * Ys + 0.024 * Xs ** 2 - 0.01 * Xs * Ys + 0.018 * Ys ** 2
    nrm = sp.sqrt(1 + sp.diff(f, Xs) ** 2 + sp.diff(f, Ys) ** 2)
    kfun = sp.lambdify((Xs, Ys), sp.diff(sp.diff(f, Xs) / nrm, Xs) +
                       sp.diff(sp.diff(f, Ys) / nrm, Ys), "numpy")
    ffun = sp.lambdify((Xs, Ys), f, "numpy")
    n, nz = 14, 18
    g = Grid(n, n, nz, h=1.0)
    s = 160
    off = (np.arange(s) + 0.5) / s
    alpha = np.zeros((nz, n, n))
    ctr = n / 2
    for j in range(n):
        for i in range(n):
            H = ffun((i + off[:, None]) - ctr, (j + off[None, :]) - ctr)
            for k in range(nz):
                alpha[k, j, i] = np.mean(np.clip(H - k, 0.0, 1.0))
    _, valid = oracle.curvature(g, alpha)
    _, faces, _ = face_kappas(g, alpha)
    checked = {0: 0, 1: 0, 2: 0}
    for d, cL, kf in faces:
        cR = right_of(d, cL, alpha.shape)
        if not (valid[cL] and valid[cR]):
            continue
        if min(cL[1], cL[2], cR[1], cR[2]) < 4 or max(cL[1], cL[2], cR[1], cR[2]) > n - 5:
            continue
        ex = 0.5 * (kfun(cL[2] + 0.5 - ctr, cL[1] + 0.5 - ctr) +
                    kfun(cR[2] + 0.5 - ctr, cR[1] + 0.5 - ctr))
        # the two column curvatures differ by more than the tolerance on x and y faces
        assert kf == pytest.approx(ex, rel=2e-3, abs=2e-5)
        checked[d] += 1
    assert checked[0] >= 3 and checked[1] >= 3 and checked[2] >= 10, checked


# --- the fallback branches, on a capped gas cylinder --------------------------------
R = 4.6
Z0, Z1 = 6.4, 18.7


def capped_cylinder():
    g = Grid(20, 20, 26, h=1.0)
    s = 64
    off = (np.arange(s) + 0.5) / s
    cx, cy = 10.3, 9.8
    xs = np.arange(g.nx)[:, None] + off[None, :] - cx
    ys = np.arange(g.ny)[:, None] + off[None, :] - cy
    inside = (xs[None, :, None, :] ** 2 + ys[:, None, :, None] ** 2) < R * R
    area = inside.mean(axis=(2, 3))  # (ny, nx)
    kz = np.arange(g.nz)
    length = np.clip(np.minimum(kz + 1, Z1) - np.maximum(kz, Z0), 0, 1)
    alpha = 1.0 - length[:, None, None] * area[None, :, :]
    # a gas pocket of 2 x 2 x 2 whole cells, away from the cylinder: no cell
    # near its faces is an interface cell, so its faces carry 0
    alpha[2:4, 15:17, 1:3] = 0.0
    return g, alpha, (cx, cy)


def block_mean(kap, valid, d, cL):
    """Mean over the valid cells of the 2 x 3 x 3 block around the face
    (cells beyond the x and y walls are not part of it)."""
    nz, ny, nx = kap.shape
    t = [a for a in range(3) if a != d]
    vals = []
    for side in (0, 1):
        for p in (-1, 0, 1):
            for q in (-1, 0, 1):
                x = [cL[2], cL[1], cL[0]]  # i, j, k
                x[d] += side
                x[t[0]] += p
                x[t[1]] += q
                if not (0 <= x[0] < nx and 0 <= x[1] < ny):
                    continue
                c = (x[2] % nz, x[1], x[0])
                if valid[c]:
                    vals.append(kap[c])
    return (sum(vals) / len(vals) if vals else 0.0), len(vals)


def test_face_curvature_branches_on_a_capped_cylinder():
    g, alpha, (cx, cy) = capped_cylinder()
    kap_c, valid = oracle.curvature(g, alpha)
    kap, faces, rep = face_kappas(g, alpha)
    assert np.array_equal(kap, kap_c)
    count = {"both": 0, "one": 0, "block": 0, "none": 0}
    for d, cL, kf in faces:
        cR = right_of(d, cL, alpha.shape)
        vL, vR = bool(valid[cL]), bool(valid[cR])
        if vL and vR:
            assert kf == 0.5 * (kap[cL] + kap[cR])
            count["both"] += 1
        elif vL or vR:
            assert kf == (kap[cL] if vL else kap[cR])
            count["one"] += 1
        else:
            ex, nvalid = block_mean(kap, valid, d, cL)
            assert kf == pytest.approx(ex, rel=1e-14, abs=1e-300)
            count["block" if nvalid else "none"] += 1
    assert rep["hf_fallbacks"] == count["block"] + count["none"]
    assert count["both"] >= 20 and count["one"] >= 20, count
    assert count["block"] >= 5 and count["none"] >= 5, count

    # geometry, independently of the branches: 1/R on the side, 0 on the caps
    side, cap = [], []
    for d, cL, kf in faces:
        k = cL[0]
        if d < 2 and Z0 + 3 <= k <= Z1 - 4:
            side.append(kf * R)
        if d == 2:
            r = np.hypot(cL[2] + 0.5 - cx, cL[1] + 0.5 - cy)
            if r < R - 2.5:
                cap.append(kf)
    assert len(side) >= 40 and len(cap) >= 10
    assert np.mean(np.abs(np.array(side) - 1.0)) < 0.05
    assert np.max(np.abs(np.array(side) - 1.0)) < 0.15
    assert np.all(np.array(cap) == 0.0)
