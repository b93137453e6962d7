"""FP64 CPU oracle for one projection time step of the VOF/SSF solver.

TEST INFRASTRUCTURE ONLY. Kumar & Vanka, "Large Scale GPU Based Simulations
of Turbulent Bubbly Flow in a Square Duct", Section 2 (Eqs. 1-7 and the
twelve-step solution procedure). Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package; the CUDA library
and its Python binding never do, and no code is shared between the two.

Fields are numpy float64 arrays shaped (nz, ny, nx) for cells,
(nz, ny, nx+1) for x-faces, (nz, ny+1, nx) for y-faces and (nz, ny, nx) for
z-faces (C order, x fastest), matching the layout in vof_oracle.h.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vof_oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

EPS = 1e-12  # interface threshold, the same constant as OR_EPS


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    hdr = os.path.join(_HERE, "vof_oracle.h")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-o", _SO, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("per_x", ctypes.c_int), ("per_y", ctypes.c_int)]


class Phys(ctypes.Structure):
    _fields_ = [("rho_l", ctypes.c_double), ("rho_g", ctypes.c_double),
                ("mu_l", ctypes.c_double), ("mu_g", ctypes.c_double),
                ("sigma", ctypes.c_double), ("g_z", ctypes.c_double),
                ("rho0", ctypes.c_double), ("dpdz", ctypes.c_double),
                ("conv_scheme", ctypes.c_int), ("kappa_mode", ctypes.c_int),
                ("kappa_exact", ctypes.c_double)]


class Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("b_mean", ctypes.c_double), ("vol_before", ctypes.c_double),
                ("vol_after", ctypes.c_double), ("vol_clipped", ctypes.c_double),
                ("max_div", ctypes.c_double), ("max_u", ctypes.c_double),
                ("hf_fallbacks", ctypes.c_long)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(d)
        _lib.or_plane_volume.restype = d
        _lib.or_plane_volume.argtypes = [dp, d]
        _lib.or_plane_constant.restype = d
        _lib.or_plane_constant.argtypes = [dp, d]
        _lib.or_normal.argtypes = [P(Grid), dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        _lib.or_hf_direction.argtypes = [dp]
        _lib.or_num_threads.restype = ctypes.c_int
        _lib.or_set_num_threads.argtypes = [ctypes.c_int]
    return _lib


def _grid(g) -> Grid:
    return Grid(int(g.nx), int(g.ny), int(g.nz), float(g.h), int(getattr(g, "per_x", 0)),
                int(getattr(g, "per_y", 0)))


def _phys(p) -> Phys:
    return Phys(p.rho_l, p.rho_g, p.mu_l, p.mu_g, p.sigma, p.g_z, p.rho0, p.dpdz,
                int(p.conv_scheme), int(p.kappa_mode), float(p.kappa_exact))


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def shapes(g):
    nx, ny, nz = g.nx, g.ny, g.nz
    return (nz, ny, nx), (nz, ny, nx + 1), (nz, ny + 1, nx), (nz, ny, nx)


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    """Cap the OpenMP threads of later oracle calls (timing only)."""
    lib().or_set_num_threads(int(n))


# --- geometry -----------------------------------------------------------------
def plane_volume(m, a: float) -> float:
    m = _f64(m)
    return lib().or_plane_volume(_ptr(m), float(a))


def plane_constant(m, alpha: float) -> float:
    m = _f64(m)
    return lib().or_plane_constant(_ptr(m), float(alpha))


def normal(g, alpha, i: int, j: int, k: int) -> np.ndarray:
    alpha = _f64(alpha)
    n = np.zeros(3)
    G = _grid(g)
    lib().or_normal(ctypes.byref(G), _ptr(alpha), i, j, k, _ptr(n))
    return n


def hf_direction(n) -> int:
    n = _f64(n)
    return lib().or_hf_direction(_ptr(n))


# --- steps of the method --------------------------------------------------------
def advect(g, alpha, u, v, w, dt: float, step_index: int, fluxes: bool = False):
    """Returns (alpha_new, report) or, with fluxes=True, (alpha_new, (fx, fy, fz), report)."""
    a = _f64(alpha).copy()
    _, us, vs, ws = shapes(g)
    fx, fy, fz = np.zeros(us), np.zeros(vs), np.zeros(ws)
    rep = Report()
    G = _grid(g)
    st = lib().or_advect(ctypes.byref(G), _ptr(a), _ptr(_f64(u)), _ptr(_f64(v)), _ptr(_f64(w)),
                         ctypes.c_double(dt), ctypes.c_long(step_index), _ptr(fx), _ptr(fy),
                         _ptr(fz), ctypes.byref(rep))
    if st != 0:
        raise RuntimeError(f"or_advect failed ({st})")
    return (a, (fx, fy, fz), rep.as_dict()) if fluxes else (a, rep.as_dict())


def curvature(g, alpha):
    cs = shapes(g)[0]
    a = _f64(alpha)
    kap = np.zeros(cs)
    valid = np.zeros(cs, dtype=np.uint8)
    G = _grid(g)
    lib().or_curvature(ctypes.byref(G), _ptr(a), _ptr(kap),
                       valid.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return kap, valid.astype(bool)


def ssf(g, p, alpha):
    cs, us, vs, ws = shapes(g)
    kap, sx, sy, sz = np.zeros(cs), np.zeros(us), np.zeros(vs), np.zeros(ws)
    rep = Report()
    G, Ph = _grid(g), _phys(p)
    st = lib().or_ssf(ctypes.byref(G), ctypes.byref(Ph), _ptr(_f64(alpha)), _ptr(kap), _ptr(sx),
                      _ptr(sy), _ptr(sz), ctypes.byref(rep))
    if st != 0:
        raise RuntimeError(f"or_ssf failed ({st})")
    return kap, sx, sy, sz, rep.as_dict()


def beta(g, p, alpha):
    _, us, vs, ws = shapes(g)
    bx, by, bz = np.zeros(us), np.zeros(vs), np.zeros(ws)
    G, Ph = _grid(g), _phys(p)
    st = lib().or_beta(ctypes.byref(G), ctypes.byref(Ph), _ptr(_f64(alpha)), _ptr(bx), _ptr(by),
                       _ptr(bz))
    if st != 0:
        raise RuntimeError(f"or_beta failed ({st})")
    return bx, by, bz


def apply_A(g, bx, by, bz, P):
    out = np.zeros(shapes(g)[0])
    G = _grid(g)
    st = lib().or_apply_A(ctypes.byref(G), _ptr(_f64(bx)), _ptr(_f64(by)), _ptr(_f64(bz)),
                          _ptr(_f64(P)), _ptr(out))
    if st != 0:
        raise RuntimeError(f"or_apply_A failed ({st})")
    return out


def solve(g, bx, by, bz, b, P0=None, rtol: float = 1e-12, max_iter: int = 200000):
    P = np.zeros(shapes(g)[0]) if P0 is None else _f64(P0).copy()
    rep = Report()
    G = _grid(g)
    st = lib().or_solve(ctypes.byref(G), _ptr(_f64(bx)), _ptr(_f64(by)), _ptr(_f64(bz)),
                        _ptr(_f64(b)), _ptr(P), ctypes.c_double(rtol), ctypes.c_int(max_iter),
                        ctypes.byref(rep))
    return P, rep.as_dict(), st


def predict(g, p, alpha_n, alpha_np1, uc, vc, wc, u, v, w, fx, fy, fz, dt: float):
    """Cell-centred intermediate velocity (steps 8-9)."""
    cs = shapes(g)[0]
    out = [np.zeros(cs) for _ in range(3)]
    G, Ph = _grid(g), _phys(p)
    st = lib().or_predict(ctypes.byref(G), ctypes.byref(Ph), _ptr(_f64(alpha_n)),
                          _ptr(_f64(alpha_np1)), _ptr(_f64(uc)), _ptr(_f64(vc)), _ptr(_f64(wc)),
                          _ptr(_f64(u)), _ptr(_f64(v)), _ptr(_f64(w)), _ptr(_f64(fx)),
                          _ptr(_f64(fy)), _ptr(_f64(fz)), ctypes.c_double(dt), *map(_ptr, out))
    if st != 0:
        raise RuntimeError(f"or_predict failed ({st})")
    return tuple(out)


def cell_to_face(g, uc, vc, wc):
    """Face velocities as the linear average of the two cells (step 10)."""
    _, us, vs, ws = shapes(g)
    u, v, w = np.zeros(us), np.zeros(vs), np.zeros(ws)
    G = _grid(g)
    st = lib().or_cell_to_face(ctypes.byref(G), _ptr(_f64(uc)), _ptr(_f64(vc)), _ptr(_f64(wc)),
                               _ptr(u), _ptr(v), _ptr(w))
    if st != 0:
        raise RuntimeError(f"or_cell_to_face failed ({st})")
    return u, v, w


def rhs(g, bx, by, bz, u, v, w, sx, sy, sz, dt: float):
    b = np.zeros(shapes(g)[0])
    G = _grid(g)
    st = lib().or_rhs(ctypes.byref(G), _ptr(_f64(bx)), _ptr(_f64(by)), _ptr(_f64(bz)),
                      _ptr(_f64(u)), _ptr(_f64(v)), _ptr(_f64(w)), _ptr(_f64(sx)), _ptr(_f64(sy)),
                      _ptr(_f64(sz)), ctypes.c_double(dt), _ptr(b))
    if st != 0:
        raise RuntimeError(f"or_rhs failed ({st})")
    return b


def correct(g, bx, by, bz, P, sx, sy, sz, dt: float, uc, vc, wc, u, v, w):
    uc, vc, wc, u, v, w = (_f64(x).copy() for x in (uc, vc, wc, u, v, w))
    rep = Report()
    G = _grid(g)
    st = lib().or_correct(ctypes.byref(G), _ptr(_f64(bx)), _ptr(_f64(by)), _ptr(_f64(bz)),
                          _ptr(_f64(P)), _ptr(_f64(sx)), _ptr(_f64(sy)), _ptr(_f64(sz)),
                          ctypes.c_double(dt), _ptr(uc), _ptr(vc), _ptr(wc), _ptr(u), _ptr(v),
                          _ptr(w), ctypes.byref(rep))
    if st != 0:
        raise RuntimeError(f"or_correct failed ({st})")
    return uc, vc, wc, u, v, w, rep.as_dict()


def project(g, p, alpha_np1, uhc, vhc, whc, uh, vh, wh, P0, sx, sy, sz, dt: float, rtol=1e-12,
            max_iter=200000):
    """Steps 11-12: assemble b from the face velocities, solve for P, correct
    faces and cells. Returns (uc, vc, wc, u, v, w, P, report, status)."""
    bx, by, bz = beta(g, p, alpha_np1)
    b = rhs(g, bx, by, bz, uh, vh, wh, sx, sy, sz, dt)
    P, srep, st = solve(g, bx, by, bz, b, P0, rtol, max_iter)
    uc, vc, wc, u, v, w, crep = correct(g, bx, by, bz, P, sx, sy, sz, dt, uhc, vhc, whc, uh, vh, wh)
    srep.update({k: crep[k] for k in ("max_div", "max_u")})
    return uc, vc, wc, u, v, w, P, srep, st


def step(g, p, alpha, uc, vc, wc, u, v, w, P, dt: float, step_index: int, rtol: float = 1e-12,
         max_iter: int = 200000):
    """One time step; returns (alpha, uc, vc, wc, u, v, w, P, report, status)."""
    arrs = [_f64(x).copy() for x in (alpha, uc, vc, wc, u, v, w, P)]
    rep = Report()
    G, Ph = _grid(g), _phys(p)
    st = lib().or_step(ctypes.byref(G), ctypes.byref(Ph), *map(_ptr, arrs), ctypes.c_double(dt),
                       ctypes.c_long(step_index), ctypes.c_double(rtol), ctypes.c_int(max_iter),
                       ctypes.byref(rep))
    if st < 0:
        raise RuntimeError(f"or_step failed ({st})")
    return (*arrs, rep.as_dict(), st)
