"""Seeded synthetic inputs for the duct/bubble workloads.

This module builds initial conditions only: grids, physical constants, gas
spheres as volume-fraction fields, duct velocity profiles and divergence-free
noise. It holds none of the time-step arithmetic, and both the CUDA library's
tests and the CPU oracle read the arrays it produces.

Physical setting (Kumar & Vanka, Section 4): air bubbles in water, rho_l =
1000, rho_g = 1.2 kg/m^3, mu_l = 1e-3 Pa s, sigma = 0.072 N/m, grid spacing
h = 48 mm / 192 = 0.25 mm. The gas viscosity is mu_l/55. Gravity acts along
-z, and the duct is periodic in z with no-slip walls in x and y.

Array layout (C order, x fastest): cells (nz, ny, nx); x-faces (nz, ny, nx+1);
y-faces (nz, ny+1, nx); z-faces (nz, ny, nx), z-face k lying between cells
k-1 and k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

H_PAPER = 0.048 / 192  # Section 4: 48 mm duct on 192 cells
RHO_L, RHO_G = 1000.0, 1.2
MU_L = 1e-3
MU_G = MU_L / 55.0
SIGMA = 0.072
GRAV = 9.81


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    h: float = H_PAPER
    per_x: int = 0
    per_y: int = 0

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def shapes(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return (nz, ny, nx), (nz, ny, nx + 1), (nz, ny + 1, nx), (nz, ny, nx)


@dataclass(frozen=True)
class Phys:
    rho_l: float = RHO_L
    rho_g: float = RHO_G
    mu_l: float = MU_L
    mu_g: float = MU_G
    sigma: float = SIGMA
    g_z: float = 0.0
    rho0: float = RHO_L
    dpdz: float = 0.0
    conv_scheme: int = 0  # 0 central, 1 first-order upwind
    kappa_mode: int = 0  # 0 height function, 1 exact
    kappa_exact: float = 0.0


@dataclass
class Case:
    """One workload: grid, constants and the initial state. Velocities are
    given at cell centres (uc, vc, wc) and on faces (u, v, w); the face field
    is discretely divergence-free and the cell field is its face average."""
    name: str
    grid: Grid
    phys: Phys
    alpha: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    P: np.ndarray
    dt: float
    steps: int
    centres: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    radius: float = 0.0
    notes: str = ""
    uc: np.ndarray = None
    vc: np.ndarray = None
    wc: np.ndarray = None

    def __post_init__(self):
        if self.uc is None:
            self.uc, self.vc, self.wc = face_to_cell(self.u, self.v, self.w)

    def state(self):
        """(alpha, uc, vc, wc, u, v, w, P) in the order the step functions take."""
        return (self.alpha, self.uc, self.vc, self.wc, self.u, self.v, self.w, self.P)


# ----------------------------------------------------------------------------
# gas spheres
# ----------------------------------------------------------------------------
def sphere_alpha(grid: Grid, centres, radius: float, sub: int = 8) -> np.ndarray:
    """Liquid fraction with gas spheres (non-overlapping, periodic in z).

    Cells wholly inside/outside a sphere are classified from their nearest
    and farthest points; cut cells use a sub x sub midpoint rule in (x, y)
    with the exact chord length in z (error well below 1e-3 per cell).
    """
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    alpha = np.ones((nz, ny, nx))
    r = float(radius)
    off = (np.arange(sub) + 0.5) / sub
    for c in np.asarray(centres, dtype=np.float64).reshape(-1, 3):
        cx, cy, cz = c
        i0, i1 = max(int(math.floor((cx - r) / h)), 0), min(int(math.floor((cx + r) / h)), nx - 1)
        j0, j1 = max(int(math.floor((cy - r) / h)), 0), min(int(math.floor((cy + r) / h)), ny - 1)
        k0, k1 = int(math.floor((cz - r) / h)), int(math.floor((cz + r) / h))
        ii = np.arange(i0, i1 + 1)
        jj = np.arange(j0, j1 + 1)
        kk = np.arange(k0, k1 + 1)  # unwrapped
        K, J, I = np.meshgrid(kk, jj, ii, indexing="ij")
        x0, y0, z0 = I * h, J * h, K * h
        dx = np.maximum(np.maximum(x0 - cx, cx - (x0 + h)), 0.0)
        dy = np.maximum(np.maximum(y0 - cy, cy - (y0 + h)), 0.0)
        dz = np.maximum(np.maximum(z0 - cz, cz - (z0 + h)), 0.0)
        dmin2 = dx * dx + dy * dy + dz * dz
        fx = np.maximum(np.abs(x0 - cx), np.abs(x0 + h - cx))
        fy = np.maximum(np.abs(y0 - cy), np.abs(y0 + h - cy))
        fz = np.maximum(np.abs(z0 - cz), np.abs(z0 + h - cz))
        dmax2 = fx * fx + fy * fy + fz * fz
        gas = np.where(dmax2 <= r * r, 1.0, 0.0)
        cut = (dmin2 < r * r) & (dmax2 > r * r)
        if np.any(cut):
            X0, Y0, Z0 = x0[cut], y0[cut], z0[cut]
            xs = X0[:, None, None] + off[None, :, None] * h
            ys = Y0[:, None, None] + off[None, None, :] * h
            q = r * r - (xs - cx) ** 2 - (ys - cy) ** 2
            half = np.sqrt(np.maximum(q, 0.0))
            lo = np.maximum(cz - half, Z0[:, None, None])
            hi = np.minimum(cz + half, Z0[:, None, None] + h)
            gas[cut] = np.mean(np.maximum(hi - lo, 0.0) / h, axis=(1, 2))
        alpha[np.mod(K, nz), J, I] -= gas
    return np.clip(alpha, 0.0, 1.0)


def place_spheres(grid: Grid, n: int, d: float, seed: int, gap: float = None,
                  wall_gap: float = None, max_tries: int = 2_000_000,
                  allow_fewer: bool = False) -> np.ndarray:
    """Seeded rejection sampling of n sphere centres (metres): centre spacing
    >= d + gap (periodic in z), and >= d/2 + wall_gap from the x/y walls.
    With allow_fewer, returns the spheres placed within max_tries instead of
    raising."""
    h = grid.h
    gap = 2 * h if gap is None else gap
    wall_gap = h if wall_gap is None else wall_gap
    W, Wy, L = grid.nx * h, grid.ny * h, grid.nz * h
    rng = np.random.default_rng(seed)
    lo = d / 2 + wall_gap
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            if allow_fewer and out:
                break
            raise RuntimeError(f"could not place {n} spheres (placed {len(out)})")
        c = np.array([rng.uniform(lo, W - lo), rng.uniform(lo, Wy - lo), rng.uniform(0, L)])
        if out:
            P = np.asarray(out)
            dz = np.abs(P[:, 2] - c[2])
            dz = np.minimum(dz, L - dz)
            dist2 = (P[:, 0] - c[0]) ** 2 + (P[:, 1] - c[1]) ** 2 + dz ** 2
            if np.any(dist2 < (d + gap) ** 2):
                continue
        out.append(c)
    return np.asarray(out)


def regular_array_centres(grid: Grid, counts=(6, 6, 24)) -> np.ndarray:
    """Bubbles on a regular array (the paper's 6 x 6 x 24 layout, Section 4)."""
    h = grid.h
    ext = (grid.nx * h, grid.ny * h, grid.nz * h)
    axes = [(np.arange(m) + 0.5) * e / m for m, e in zip(counts, ext)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


# ----------------------------------------------------------------------------
# velocity fields
# ----------------------------------------------------------------------------
def laminar_duct_profile(x, y, W: float, G: float, mu: float, nterms: int = 199):
    """Fully developed laminar flow in the square duct [0,W]^2 driven by a
    force G per volume along +z: the textbook Fourier series solution of
    mu (w_xx + w_yy) = -G with w = 0 on the walls."""
    a = W / 2.0
    X = np.asarray(x, dtype=np.float64) - a
    Y = np.abs(np.asarray(y, dtype=np.float64) - a)
    s = np.zeros(np.broadcast(X, Y).shape)
    for n in range(1, nterms + 1, 2):
        kn = n * math.pi / (2 * a)
        # cosh(kn*Y)/cosh(kn*a) written without overflow
        ratio = np.exp(kn * (Y - a)) * (1 + np.exp(-2 * kn * Y)) / (1 + math.exp(-2 * kn * a))
        s = s + ((-1) ** ((n - 1) // 2)) * (1 - ratio) * np.cos(kn * X) / n ** 3
    return 16 * G * a * a / (mu * math.pi ** 3) * s


def _face_centres(grid: Grid):
    h = grid.h
    xc = (np.arange(grid.nx) + 0.5) * h
    yc = (np.arange(grid.ny) + 0.5) * h
    return xc, yc


def laminar_w(grid: Grid, w_b: float, mu: float):
    """w on z-faces from the laminar series, scaled to the bulk velocity
    w_b; returns (w, G) with G the driving force that sustains it."""
    xc, yc = _face_centres(grid)
    prof = laminar_duct_profile(xc[None, :], yc[:, None], grid.nx * grid.h, 1.0, mu)
    G = w_b / prof.mean()
    w2 = prof * G
    return np.broadcast_to(w2, (grid.nz, grid.ny, grid.nx)).copy(), G


def power_law_w(grid: Grid, w_b: float):
    """1/7-power mean profile w = c f(x) f(y) with f(s) = (2s/W)^(1/7) folded
    about the duct centre, scaled to bulk velocity w_b (Section 4 initial
    profile, applied in both wall-normal directions)."""
    xc, yc = _face_centres(grid)
    W = grid.nx * grid.h

    def f(s):
        t = np.minimum(2 * s / W, 2 - 2 * s / W)
        return np.power(np.maximum(t, 0.0), 1.0 / 7.0)

    prof = f(xc)[None, :] * f(yc)[:, None]
    prof *= w_b / prof.mean()
    return np.broadcast_to(prof, (grid.nz, grid.ny, grid.nx)).copy()


def curl_noise(grid: Grid, rms: float, seed: int, kmax: int = 4):
    """Exactly (discretely) solenoidal face velocities: the discrete curl of
    a seeded smooth vector potential on the cell edges, with the potential's
    wall-tangential components zero so no velocity crosses a wall. Scaled so
    the RMS over all face values is `rms`."""
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    W, Wy, L = nx * h, ny * h, nz * h
    rng = np.random.default_rng(seed)
    m = np.arange(1, kmax + 1)

    def sinx(xs, ext):  # (kmax, n) modes vanishing at both walls
        return np.sin(np.pi * m[:, None] * xs[None, :] / ext)

    def zmodes(zs):  # (2*kmax, n) periodic modes
        ph = 2 * np.pi * m[:, None] * zs[None, :] / L
        return np.concatenate([np.cos(ph), np.sin(ph)], axis=0)

    xn, xc = np.arange(nx + 1) * h, (np.arange(nx) + 0.5) * h
    yn, yc = np.arange(ny + 1) * h, (np.arange(ny) + 0.5) * h
    zn, zc = np.arange(nz) * h, (np.arange(nz) + 0.5) * h

    def field3(Sx, Sy, Sz):
        coef = rng.standard_normal((Sx.shape[0], Sy.shape[0], Sz.shape[0]))
        coef /= (1 + np.arange(Sx.shape[0]))[:, None, None]
        return np.einsum("abc,ai,bj,ck->kji", coef, Sx, Sy, Sz, optimize=True)

    # Ax on edges (x centre, y node, z node); Ay (x node, y centre, z node);
    # Az (x node, y node, z centre). Tangential components vanish on walls.
    Ax = field3(np.concatenate([sinx(xc, W), np.cos(np.pi * m[:, None] * xc[None, :] / W)]),
                sinx(yn, Wy), zmodes(zn))
    Ay = field3(sinx(xn, W),
                np.concatenate([sinx(yc, Wy), np.cos(np.pi * m[:, None] * yc[None, :] / Wy)]),
                zmodes(zn))
    Az = field3(sinx(xn, W), sinx(yn, Wy), zmodes(zc))
    # Ax: (nz, ny+1, nx); Ay: (nz, ny, nx+1); Az: (nz, ny+1, nx+1)
    up = lambda A: np.roll(A, -1, axis=0)  # z + 1 (periodic)
    u = (Az[:, 1:, :] - Az[:, :-1, :]) / h - (up(Ay) - Ay) / h
    v = (up(Ax) - Ax) / h - (Az[:, :, 1:] - Az[:, :, :-1]) / h
    w = (Ay[:, :, 1:] - Ay[:, :, :-1]) / h - (Ax[:, 1:, :] - Ax[:, :-1, :]) / h
    # remove rounding noise on the wall faces (exactly zero in exact arithmetic)
    u[:, :, 0] = 0.0
    u[:, :, -1] = 0.0
    v[:, 0, :] = 0.0
    v[:, -1, :] = 0.0
    tot = np.concatenate([u.ravel(), v.ravel(), w.ravel()])
    s = rms / math.sqrt(np.mean(tot * tot))
    return u * s, v * s, w * s


def face_to_cell(u, v, w):
    """Cell-centred velocity components as the mean of the two faces."""
    return (0.5 * (u[:, :, 1:] + u[:, :, :-1]), 0.5 * (v[:, 1:, :] + v[:, :-1, :]),
            0.5 * (w + np.roll(w, -1, axis=0)))


def divergence(grid: Grid, u, v, w):
    """Discrete divergence per cell (input sanity checks only)."""
    h = grid.h
    return ((u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :]) +
            (np.roll(w, -1, axis=0) - w)) / h


def stable_dt(grid: Grid, phys: Phys, umax: float, cfl: float = 0.25, safety: float = 0.5):
    """Fixed time step: the smallest of the advective (CFL), capillary and
    explicit-viscous limits, times a safety factor. The viscous limit uses
    the largest viscosity over the smallest density, since cells at the
    interface mix the liquid's viscosity with the gas's density."""
    h = grid.h
    lims = []
    if phys.sigma > 0:
        lims.append(math.sqrt((phys.rho_l + phys.rho_g) * h ** 3 / (4 * math.pi * phys.sigma)))
    nu = max(phys.mu_l, phys.mu_g) / min(phys.rho_l, phys.rho_g)
    if nu > 0:
        lims.append(h * h / (6 * nu))
    if umax > 0:
        lims.append(cfl * h / umax)
    return safety * min(lims)


def gas_fraction(alpha) -> float:
    return float(1.0 - np.mean(alpha))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
def static_bubble(n: int = 32, radius_cells: float = 8.0, kappa_mode: int = 0,
                  steps: int = 20) -> Case:
    """Static gas bubble of radius 8h centred in a 32^3 periodic-z duct, zero
    velocity, no gravity: the Laplace-balance test (Section 2.1, the claim
    that spurious currents vanish with exact curvature)."""
    g = Grid(n, n, n)
    R = radius_cells * g.h
    centre = np.array([[n / 2 * g.h] * 3])
    alpha = sphere_alpha(g, centre, R)
    ph = Phys(kappa_mode=kappa_mode, kappa_exact=2.0 / R)
    cs, us, vs, ws = g.shapes()
    dt = stable_dt(g, ph, 0.0)
    return Case("static_bubble", g, ph, alpha, np.zeros(us), np.zeros(vs), np.zeros(ws),
                np.zeros(cs), dt, steps, centre, R,
                "32^3, one sphere R=8h centred, zero velocity, no gravity")


def rising_swarm(nx: int = 64, ny: int = 64, nz: int = 128, nbub: int = 8, d_cells: float = 12,
                 seed: int = 2104, steps: int = 200, w_b: float = 0.1104) -> Case:
    """Bubbles in laminar duct flow plus divergence-free noise at 10% of the
    bulk velocity, gravity along -z."""
    g = Grid(nx, ny, nz)
    d = d_cells * g.h
    centres = place_spheres(g, nbub, d, seed)
    c = _swarm_from(g, centres, d, seed, steps, w_b)
    c.name = "rising_swarm"
    c.notes = f"{nx}x{ny}x{nz}, {nbub} spheres d={d_cells}h, laminar w_b={w_b} + 10% noise"
    return c


def paper_shaped(nx: int = 224, ny: int = 224, nz: int = 640, nbub: int = 864,
                 d_cells: float = 12, seed: int = 2106, regular: bool = False,
                 steps: int = 50) -> Case:
    """Paper-shaped duct: ~32.1M cells, 864 spheres of d = 12h, 1/7-power
    mean profile at Re_b = 5300 plus 8% divergence-free perturbations
    (Section 4), driving force from Re_tau = 360."""
    g = Grid(nx, ny, nz)
    d = d_cells * g.h
    W = nx * g.h
    centres = (regular_array_centres(g) if regular else place_spheres(g, nbub, d, seed))
    alpha = sphere_alpha(g, centres, d / 2)
    w_b = 5300 * MU_L / (RHO_L * W)
    u_tau = 360 * MU_L / (RHO_L * W)
    dpdz = 4 * RHO_L * u_tau ** 2 / W
    un, vn, wn = curl_noise(g, 0.08 * w_b, seed + 1, kmax=3)
    phi = gas_fraction(alpha)
    ph = Phys(g_z=-GRAV, rho0=(1 - phi) * RHO_L + phi * RHO_G, dpdz=dpdz)
    u, v, w = un, vn, power_law_w(g, w_b) + wn
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    cs = g.shapes()[0]
    return Case("paper_shaped", g, ph, alpha, u, v, w, np.zeros(cs), stable_dt(g, ph, umax),
                steps, centres, d / 2,
                f"{nx}x{ny}x{nz}, {len(centres)} spheres d={d_cells}h, 1/7 profile Re_b=5300")


def with_phys(case: Case, **kw) -> Case:
    return replace(case, phys=replace(case.phys, **kw))


# ----------------------------------------------------------------------------
# request mix for the serving loop
# ----------------------------------------------------------------------------
SERVE_GRIDS = ((32, 32, 32), (64, 64, 128), (96, 96, 192), (128, 128, 256))


@dataclass
class Request:
    kind: str          # "step" (n_steps time steps) or "solve" (one pressure solve)
    case: Case
    n_steps: int
    b: np.ndarray = None  # right side of a solve


def serving_mix(n_req: int, seed: int = 2108, grids=SERVE_GRIDS, p_step: float = 0.5):
    """Seeded request mix: grid drawn uniformly from `grids`, 1-64 spheres
    with d drawn from [8, 14]h (fewer where the grid cannot hold them), the
    rising-swarm flow, and either 1-10 time steps or one pressure solve whose
    right side is zero-mean Gaussian noise scaled like -div(u)/dt of the
    case's flow. The paper has no serving workload; this stands in for an
    ensemble of independent duct cases."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_req):
        dims = grids[int(rng.integers(len(grids)))]
        d_cells = float(rng.uniform(8.0, 14.0))
        nbub = int(rng.integers(1, 65))
        kind = "step" if rng.uniform() < p_step else "solve"
        n_steps = int(rng.integers(1, 11)) if kind == "step" else 0
        sub = seed * 1000 + r
        g = Grid(*dims)
        d = d_cells * g.h
        centres = place_spheres(g, nbub, d, sub, max_tries=20_000, allow_fewer=True)
        case = _swarm_from(g, centres, d, sub, max(n_steps, 1))
        b = None
        if kind == "solve":
            b = np.random.default_rng(sub + 1).normal(size=g.shapes()[0])
            b = (b - b.mean()) * (0.1 * 0.1104 / g.h / case.dt)
        out.append(Request(kind, case, n_steps, b))
    return out


def _swarm_from(g: Grid, centres, d: float, seed: int, steps: int, w_b: float = 0.1104) -> Case:
    """Rising-swarm flow (laminar duct profile of bulk velocity w_b + 10%
    divergence-free noise, gravity along -z) around the given sphere centres."""
    alpha = sphere_alpha(g, centres, d / 2)
    w0, G = laminar_w(g, w_b, MU_L)
    un, vn, wn = curl_noise(g, 0.10 * w_b, seed + 1)
    phi = gas_fraction(alpha)
    ph = Phys(g_z=-GRAV, rho0=(1 - phi) * RHO_L + phi * RHO_G, dpdz=G)
    u, v, w = un, vn, w0 + wn
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    return Case("serve", g, ph, alpha, u, v, w, np.zeros(g.shapes()[0]),
                stable_dt(g, ph, umax), steps, centres, d / 2)


def ensemble_cases(n: int = 64, dims=(48, 48, 96), seed: int = 2109):
    """n independent small ducts of one grid size: per case 4-16 spheres with
    d drawn from [8, 14]h (fewer where they do not fit) in the rising-swarm
    flow. The paper has no ensemble workload; this is the seeded stand-in for
    a batch of independent cases."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        g = Grid(*dims)
        d = float(rng.uniform(8.0, 14.0)) * g.h
        nbub = int(rng.integers(4, 17))
        sub = seed * 1000 + c
        centres = place_spheres(g, nbub, d, sub, max_tries=20_000, allow_fewer=True)
        case = _swarm_from(g, centres, d, sub, 1)
        case.name = "ensemble"
        out.append(case)
    return out
