/*
 * vof_oracle.c -- plain FP64 CPU oracle for one projection time step of the
 * air-water VOF / sharp-surface-force solver (Kumar & Vanka, Section 2).
 *
 * TEST INFRASTRUCTURE ONLY (see vof_oracle.h). Written for obviousness, not
 * speed: every quantity is recomputed from its definition at the point of
 * use, loops follow the paper's order of operations, and the only
 * parallelism is an OpenMP split over z-planes whose partial sums are
 * combined in plane order (results do not depend on the thread count).
 *
 * Readings of the paper that this file implements (the paper is silent or
 * garbled on them; the CUDA library follows the same readings):
 *  - velocities live at cell centres (the momentum variable, Section 2:
 *    a collocated grid) and on cell faces (the divergence-free field that
 *    advects alpha); face values are the linear average of the two cells
 *    (step 10) corrected by the face pressure gradient (steps 11-12), and the
 *    cells are corrected by the average of their two face corrections;
 *  - momentum is convected with the mass fluxes of the geometric VOF sweep
 *    (step 9: sum over phases of rho_k times the phase volume flux), with
 *    the donor cell's velocity (upwind) or the two-cell mean (central);
 *  - the interface normal is minus the central gradient of alpha smoothed
 *    with the separable [1,2,1]^3/64 kernel (Section 2, Rudman smoothing);
 *  - geometric donor-slab fluxes with direction splitting, x-y-z on even
 *    steps and z-y-x on odd steps, with the divergence term weighted by
 *    c = [alpha^n > 1/2] frozen over the three sweeps (Section 2.1, the
 *    "second-order operator split" of Eq. 3);
 *  - height-function curvature from 7-cell column sums (Section 2, Cummins);
 *  - the sharp surface force s_f = sigma kappa_f (G_R - G_L)/h with the gas
 *    indicator G = [alpha < 1/2] (Eq. 6), and the pressure jump enters the
 *    single combined pressure P = p + p_tilde (Eqs. 6-7 and step 11 are
 *    linear in the source, so one solve equals the two of steps 6 and 11);
 *  - linear face averaging rho_f = (rho_L + rho_R)/2 (step 10), beta = 1/rho_f.
 *
 * Every step is pinned by CPU tests against something other than this file:
 * exact rational volumes, closed-form eigenvalues and series, the symbolic
 * curvature of quadric surfaces, polynomial fields on which the stencils are
 * exact (the viscous full stress, walls included), brute-force enumeration
 * and conservation invariants. The viscous term and the face curvature are
 * also checked by planting mistakes in a copy of this file
 * (tests/test_oracle_mutants.py). Only the size of the spurious currents
 * with height-function curvature is not fixed by the paper (reported, not
 * pinned).
 */
#include "vof_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* indexing                                                                  */
/* ------------------------------------------------------------------------ */
static inline int wrapi(int i, int n) { i %= n; return i < 0 ? i + n : i; }
static inline long C_(const or_grid* g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)wrapi(k, g->nz));
}
static inline long U_(const or_grid* g, int i, int j, int k) {
    return (long)i + (long)(g->nx + 1) * ((long)j + (long)g->ny * (long)wrapi(k, g->nz));
}
static inline long V_(const or_grid* g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)(g->ny + 1) * (long)wrapi(k, g->nz));
}
static inline long W_(const or_grid* g, int i, int j, int k) {
    return (long)i + (long)g->nx * ((long)j + (long)g->ny * (long)wrapi(k, g->nz));
}
static inline long ncells(const or_grid* g) { return (long)g->nx * g->ny * g->nz; }

/* alpha with the boundary ghosts: walls are wetted (ghost alpha = 1,
 * Section 5 footnote on complete wetting); periodic directions wrap. */
static double alpha_at(const or_grid* g, const double* a, int i, int j, int k) {
    if (g->per_x) i = wrapi(i, g->nx);
    else if (i < 0 || i >= g->nx) return 1.0;
    if (g->per_y) j = wrapi(j, g->ny);
    else if (j < 0 || j >= g->ny) return 1.0;
    return a[C_(g, i, j, k)];
}

/* Sum in z-plane order of per-plane partial sums. */
static double ordered_sum(const double* part, int nz) {
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += part[k];
    return s;
}

/* ------------------------------------------------------------------------ */
/* PLIC geometry                                                             */
/* ------------------------------------------------------------------------ */
/* Length of {z in [0,1] : mz*z <= t}. */
static double seg_len(double mz, double t) {
    if (mz > 0.0) {
        double s = t / mz;
        return s <= 0.0 ? 0.0 : (s >= 1.0 ? 1.0 : s);
    }
    if (mz < 0.0) {
        double s = t / mz; /* the set is z >= s */
        return s <= 0.0 ? 1.0 : (s >= 1.0 ? 0.0 : 1.0 - s);
    }
    return t >= 0.0 ? 1.0 : 0.0;
}

static void sort_small(double* b, int n) {
    for (int i = 1; i < n; ++i)
        for (int j = i; j > 0 && b[j - 1] > b[j]; --j) {
            double t = b[j]; b[j] = b[j - 1]; b[j - 1] = t;
        }
}

/* Area of {(y,z) in [0,1]^2 : my*y + mz*z <= c}: seg_len is linear in y
 * between its two kinks, so the midpoint rule on each piece is exact. */
static double strip_area(double my, double mz, double c) {
    double br[4];
    int nb = 0;
    br[nb++] = 0.0;
    if (my != 0.0) {
        double y1 = c / my, y2 = (c - mz) / my;
        if (y1 > 0.0 && y1 < 1.0) br[nb++] = y1;
        if (y2 > 0.0 && y2 < 1.0) br[nb++] = y2;
    }
    br[nb++] = 1.0;
    sort_small(br, nb);
    double s = 0.0;
    for (int p = 0; p + 1 < nb; ++p) {
        double len = br[p + 1] - br[p];
        if (len <= 0.0) continue;
        s += len * seg_len(mz, c - my * 0.5 * (br[p] + br[p + 1]));
    }
    return s;
}

/* Volume of the part of the unit cube below the plane m.xi = a. The strip
 * area is a piecewise quadratic in x with kinks where c = a - mx*x crosses
 * 0, my, mz, my+mz; two-point Gauss-Legendre on each piece is exact. The
 * axis with the largest |m| is integrated first so no division is by a
 * small component. */
double or_plane_volume(const double m_in[3], double a) {
    int big = 0;
    if (fabs(m_in[1]) > fabs(m_in[big])) big = 1;
    if (fabs(m_in[2]) > fabs(m_in[big])) big = 2;
    double mz = m_in[big];
    double mx = m_in[(big + 1) % 3], my = m_in[(big + 2) % 3];
    double br[6];
    int nb = 0;
    br[nb++] = 0.0;
    if (mx != 0.0) {
        const double kinks[4] = {0.0, my, mz, my + mz};
        for (int q = 0; q < 4; ++q) {
            double x = (a - kinks[q]) / mx;
            if (x > 0.0 && x < 1.0) br[nb++] = x;
        }
    }
    br[nb++] = 1.0;
    sort_small(br, nb);
    const double gl = 0.57735026918962576451; /* 1/sqrt(3) */
    double vol = 0.0;
    for (int p = 0; p + 1 < nb; ++p) {
        double half = 0.5 * (br[p + 1] - br[p]);
        if (half <= 0.0) continue;
        double mid = 0.5 * (br[p + 1] + br[p]);
        double x1 = mid - half * gl, x2 = mid + half * gl;
        vol += half * (strip_area(my, mz, a - mx * x1) + strip_area(my, mz, a - mx * x2));
    }
    return vol;
}

/* Plane constant by bisection on the monotone volume function. */
double or_plane_constant(const double m[3], double alpha) {
    double lo = 0.0, hi = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (m[d] < 0.0) lo += m[d]; else hi += m[d];
    }
    if (alpha <= 0.0) return lo;
    if (alpha >= 1.0) return hi;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (or_plane_volume(m, mid) < alpha) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Smoothed alpha: separable [1,2,1] weights in each direction, sum 64. */
static double alpha_smooth(const or_grid* g, const double* a, int i, int j, int k) {
    static const double wt[3] = {1.0, 2.0, 1.0};
    double s = 0.0;
    for (int c = -1; c <= 1; ++c)
        for (int b = -1; b <= 1; ++b)
            for (int q = -1; q <= 1; ++q)
                s += wt[q + 1] * wt[b + 1] * wt[c + 1] * alpha_at(g, a, i + q, j + b, k + c);
    return s / 64.0;
}

/* Interface normal in cell units: minus the central difference of the
 * smoothed alpha, so it points from liquid into gas and the liquid lies on
 * the side n.xi <= d of the plane. */
void or_normal(const or_grid* g, const double* a, int i, int j, int k, double n[3]) {
    n[0] = -(alpha_smooth(g, a, i + 1, j, k) - alpha_smooth(g, a, i - 1, j, k)) / 2.0;
    n[1] = -(alpha_smooth(g, a, i, j + 1, k) - alpha_smooth(g, a, i, j - 1, k)) / 2.0;
    n[2] = -(alpha_smooth(g, a, i, j, k + 1) - alpha_smooth(g, a, i, j, k - 1)) / 2.0;
}

/* argmax |n_d| with ties (within a relative 1e-9) going to the lower axis,
 * so that rounding differences cannot flip the choice. */
int or_hf_direction(const double n[3]) {
    int d = 0;
    double best = fabs(n[0]);
    if (fabs(n[1]) > best * (1.0 + 1e-9)) { d = 1; best = fabs(n[1]); }
    if (fabs(n[2]) > best * (1.0 + 1e-9)) { d = 2; }
    return d;
}

static int is_interface(double a) { return a > OR_EPS && a < 1.0 - OR_EPS; }

/* ------------------------------------------------------------------------ */
/* VOF advection                                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    unsigned char* has; /* cell carries a plane */
    double* n;          /* 3 per cell */
    double* d;          /* plane constant */
} plic_t;

static void reconstruct(const or_grid* g, const double* a, plic_t* P) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long c = C_(g, i, j, k);
                P->has[c] = 0;
                P->d[c] = 0.0;
                P->n[3 * c] = P->n[3 * c + 1] = P->n[3 * c + 2] = 0.0;
                if (!is_interface(a[c])) continue;
                double n[3];
                or_normal(g, a, i, j, k, n);
                if (n[0] == 0.0 && n[1] == 0.0 && n[2] == 0.0) continue;
                P->has[c] = 1;
                P->n[3 * c] = n[0]; P->n[3 * c + 1] = n[1]; P->n[3 * c + 2] = n[2];
                P->d[c] = or_plane_constant(n, a[c]);
            }
}

/* Signed liquid volume (in cell volumes) crossing a face of direction dir
 * whose left (-) cell is cL and right (+) cell is cR, in one sweep: the
 * liquid inside the donor-cell slab of width |vel|*dt adjacent to the face
 * (Rider-Kothe geometric construction). Cells without a plane flux their
 * uniform content. */
static double face_flux(const or_grid* g, const double* a, const plic_t* P, int dir,
                        long cL, long cR, double vel, double dt) {
    if (vel == 0.0) return 0.0;
    double c = fabs(vel) * dt / g->h;
    long dn = vel > 0.0 ? cL : cR;
    double vol;
    if (!P->has[dn]) {
        vol = c * a[dn];
    } else {
        double m[3] = {P->n[3 * dn], P->n[3 * dn + 1], P->n[3 * dn + 2]};
        double d = P->d[dn];
        if (vel > 0.0) d -= m[dir] * (1.0 - c); /* slab xi_dir in [1-c, 1] */
        m[dir] *= c;                            /* rescale the slab to a unit cube */
        vol = c * or_plane_volume(m, d);
    }
    return vel > 0.0 ? vol : -vol;
}

/* Face velocity and donor/acceptor cells on the minus (side=0) or plus
 * (side=1) face of cell (i,j,k) in direction dir. Returns 0 and vel=0 at a
 * wall face. */
static int face_of(const or_grid* g, const double* u, const double* v, const double* w,
                   int dir, int side, int i, int j, int k, long* cL, long* cR, double* vel) {
    int ii = i, jj = j, kk = k;
    if (dir == 0) {
        int f = i + side; /* face index */
        if (!g->per_x && (f == 0 || f == g->nx)) { *vel = 0.0; return 0; }
        int fw = wrapi(f, g->nx);
        *vel = u[U_(g, fw, j, k)];
        *cL = C_(g, wrapi(f - 1, g->nx), jj, kk);
        *cR = C_(g, fw, jj, kk);
    } else if (dir == 1) {
        int f = j + side;
        if (!g->per_y && (f == 0 || f == g->ny)) { *vel = 0.0; return 0; }
        int fw = wrapi(f, g->ny);
        *vel = v[V_(g, i, fw, k)];
        *cL = C_(g, ii, wrapi(f - 1, g->ny), kk);
        *cR = C_(g, ii, fw, kk);
    } else {
        int f = wrapi(k + side, g->nz);
        *vel = w[W_(g, i, j, f)];
        *cL = C_(g, ii, jj, f - 1);
        *cR = C_(g, ii, jj, f);
    }
    return 1;
}

int or_advect(const or_grid* g, double* alpha, const double* u, const double* v,
              const double* w, double dt, long step_index, double* fx, double* fy, double* fz,
              or_report* rep) {
    long N = ncells(g);
    double h3 = g->h * g->h * g->h;
    unsigned char* cm = (unsigned char*)malloc((size_t)N);
    double* anew = (double*)malloc(sizeof(double) * (size_t)N);
    double* part = (double*)calloc((size_t)g->nz, sizeof(double));
    double* cpart = (double*)calloc((size_t)g->nz, sizeof(double));
    plic_t P;
    P.has = (unsigned char*)malloc((size_t)N);
    P.n = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    P.d = (double*)malloc(sizeof(double) * (size_t)N);
    if (!cm || !anew || !part || !cpart || !P.has || !P.n || !P.d) return -2;

    /* liquid volume before; frozen divergence weight c = [alpha^n > 1/2] */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        double s = 0.0;
        for (long c = (long)k * g->nx * g->ny; c < (long)(k + 1) * g->nx * g->ny; ++c) {
            s += alpha[c];
            cm[c] = alpha[c] > 0.5;
        }
        part[k] = s;
    }
    double vol_before = ordered_sum(part, g->nz) * h3;

    double* fl[3] = {fx, fy, fz};
    const long nface[3] = {(long)(g->nx + 1) * g->ny * g->nz, (long)g->nx * (g->ny + 1) * g->nz, N};
    for (int d = 0; d < 3; ++d)
        if (fl[d]) memset(fl[d], 0, sizeof(double) * (size_t)nface[d]);
    for (int s = 0; s < 3; ++s) {
        int dir = (step_index % 2 == 0) ? s : 2 - s;
        reconstruct(g, alpha, &P);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < g->nz; ++k) {
            double clip = 0.0;
            for (int j = 0; j < g->ny; ++j)
                for (int i = 0; i < g->nx; ++i) {
                    long c = C_(g, i, j, k);
                    long L, R;
                    double vm, vp, fm = 0.0, fp = 0.0;
                    if (face_of(g, u, v, w, dir, 0, i, j, k, &L, &R, &vm))
                        fm = face_flux(g, alpha, &P, dir, L, R, vm, dt);
                    /* record the flux of this face (each face is the minus face of one cell) */
                    if (fl[dir]) {
                        if (dir == 0) fl[0][U_(g, i, j, k)] = fm;
                        else if (dir == 1) fl[1][V_(g, i, j, k)] = fm;
                        else fl[2][W_(g, i, j, k)] = fm;
                    }
                    if (face_of(g, u, v, w, dir, 1, i, j, k, &L, &R, &vp))
                        fp = face_flux(g, alpha, &P, dir, L, R, vp, dt);
                    double an = alpha[c] - (fp - fm) + (cm[c] ? 1.0 : 0.0) * (vp - vm) * dt / g->h;
                    double ac = an < 0.0 ? 0.0 : (an > 1.0 ? 1.0 : an);
                    clip += an - ac;
                    anew[c] = ac;
                }
            cpart[k] = clip;
        }
        memcpy(alpha, anew, sizeof(double) * (size_t)N);
        if (rep) rep->vol_clipped += ordered_sum(cpart, g->nz) * h3;
    }

#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        double s = 0.0;
        for (long c = (long)k * g->nx * g->ny; c < (long)(k + 1) * g->nx * g->ny; ++c) s += alpha[c];
        part[k] = s;
    }
    if (rep) {
        rep->vol_before = vol_before;
        rep->vol_after = ordered_sum(part, g->nz) * h3;
    }
    free(cm); free(anew); free(part); free(cpart); free(P.has); free(P.n); free(P.d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Height-function curvature and the sharp surface force                     */
/* ------------------------------------------------------------------------ */
/* Curvature at an interface cell from the 3x3 block of 7-cell column sums
 * along the dominant normal direction. kappa is the divergence of the unit
 * normal that points into the liquid, so a gas sphere of radius R has
 * kappa = 2/R; written with the liquid column sums this formula holds for
 * either orientation of the column. Returns 1 when every column starts and
 * ends in opposite phases. */
static int hf_kappa(const or_grid* g, const double* a, int i, int j, int k, double* kap) {
    double n[3];
    or_normal(g, a, i, j, k, n);
    int d = or_hf_direction(n);
    int t1 = d == 0 ? 1 : 0;
    int t2 = d == 2 ? 1 : 2;
    double col[3][3];
    int ok = 1;
    for (int p = -1; p <= 1; ++p)
        for (int q = -1; q <= 1; ++q) {
            double s = 0.0, a_lo = 0.0, a_hi = 0.0;
            for (int r = -3; r <= 3; ++r) {
                int o[3] = {0, 0, 0};
                o[d] = r; o[t1] = p; o[t2] = q;
                double av = alpha_at(g, a, i + o[0], j + o[1], k + o[2]);
                s += av;
                if (r == -3) a_lo = av;
                if (r == 3) a_hi = av;
            }
            col[p + 1][q + 1] = s;
            if ((a_lo >= 0.5) == (a_hi >= 0.5)) ok = 0;
        }
    double H1 = (col[2][1] - col[0][1]) / 2.0;
    double H2 = (col[1][2] - col[1][0]) / 2.0;
    double H11 = col[2][1] - 2.0 * col[1][1] + col[0][1];
    double H22 = col[1][2] - 2.0 * col[1][1] + col[1][0];
    double H12 = (col[2][2] - col[2][0] - col[0][2] + col[0][0]) / 4.0;
    double den = 1.0 + H1 * H1 + H2 * H2;
    *kap = (H11 * (1.0 + H2 * H2) + H22 * (1.0 + H1 * H1) - 2.0 * H12 * H1 * H2) /
           (g->h * den * sqrt(den));
    return ok;
}

int or_curvature(const or_grid* g, const double* alpha, double* kappa, unsigned char* valid) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long c = C_(g, i, j, k);
                double kap = 0.0;
                int ok = 0;
                if (is_interface(alpha[c])) ok = hf_kappa(g, alpha, i, j, k, &kap);
                kappa[c] = ok ? kap : 0.0;
                if (valid) valid[c] = (unsigned char)ok;
            }
    return 0;
}

/* Face curvature: mean of the valid cell values on either side, else the
 * mean over the valid cells of the 2x3x3 block around the face, else 0. */
static double face_kappa(const or_grid* g, const double* kappa, const unsigned char* valid,
                         int dir, int iL, int jL, int kL, long* fallbacks) {
    int o[3] = {0, 0, 0};
    o[dir] = 1;
    long cL = C_(g, iL, jL, kL), cR = C_(g, iL + o[0], jL + o[1], kL + o[2]);
    if (valid[cL] && valid[cR]) return 0.5 * (kappa[cL] + kappa[cR]);
    if (valid[cL]) return kappa[cL];
    if (valid[cR]) return kappa[cR];
    int t1 = dir == 0 ? 1 : 0, t2 = dir == 2 ? 1 : 2;
    double s = 0.0;
    int cnt = 0;
    for (int side = 0; side <= 1; ++side)
        for (int p = -1; p <= 1; ++p)
            for (int q = -1; q <= 1; ++q) {
                int x[3] = {iL, jL, kL};
                x[dir] += side; x[t1] += p; x[t2] += q;
                if (x[0] < 0 || x[0] >= g->nx || x[1] < 0 || x[1] >= g->ny) continue;
                long c = C_(g, x[0], x[1], x[2]);
                if (valid[c]) { s += kappa[c]; ++cnt; }
            }
    (*fallbacks)++;
    return cnt ? s / cnt : 0.0;
}

int or_ssf(const or_grid* g, const or_phys* p, const double* alpha, double* kappa,
           double* sx, double* sy, double* sz, or_report* rep) {
    if (g->per_x || g->per_y) return -1;
    long N = ncells(g);
    unsigned char* valid = (unsigned char*)malloc((size_t)N);
    long* fb = (long*)calloc((size_t)g->nz, sizeof(long));
    if (!valid || !fb) return -2;
    if (p->kappa_mode == 1) {
        for (long c = 0; c < N; ++c) {
            valid[c] = (unsigned char)is_interface(alpha[c]);
            kappa[c] = valid[c] ? p->kappa_exact : 0.0;
        }
    } else {
        or_curvature(g, alpha, kappa, valid);
    }
    const int nx = g->nx, ny = g->ny, nz = g->nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        long nfb = 0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                double s = 0.0;
                if (i > 0 && i < nx) {
                    double GL = alpha[C_(g, i - 1, j, k)] < 0.5, GR = alpha[C_(g, i, j, k)] < 0.5;
                    if (GL != GR) {
                        double kf = p->kappa_mode == 1 ? p->kappa_exact
                                                       : face_kappa(g, kappa, valid, 0, i - 1, j, k, &nfb);
                        s = p->sigma * kf * (GR - GL) / g->h;
                    }
                }
                sx[U_(g, i, j, k)] = s;
            }
        for (int j = 0; j <= ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = 0.0;
                if (j > 0 && j < ny) {
                    double GL = alpha[C_(g, i, j - 1, k)] < 0.5, GR = alpha[C_(g, i, j, k)] < 0.5;
                    if (GL != GR) {
                        double kf = p->kappa_mode == 1 ? p->kappa_exact
                                                       : face_kappa(g, kappa, valid, 1, i, j - 1, k, &nfb);
                        s = p->sigma * kf * (GR - GL) / g->h;
                    }
                }
                sy[V_(g, i, j, k)] = s;
            }
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = 0.0;
                double GL = alpha[C_(g, i, j, k - 1)] < 0.5, GR = alpha[C_(g, i, j, k)] < 0.5;
                if (GL != GR) {
                    double kf = p->kappa_mode == 1 ? p->kappa_exact
                                                   : face_kappa(g, kappa, valid, 2, i, j, k - 1, &nfb);
                    s = p->sigma * kf * (GR - GL) / g->h;
                }
                sz[W_(g, i, j, k)] = s;
            }
        fb[k] = nfb;
    }
    if (rep) {
        long t = 0;
        for (int k = 0; k < nz; ++k) t += fb[k];
        rep->hf_fallbacks += t;
    }
    free(valid); free(fb);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Mixture properties                                                        */
/* ------------------------------------------------------------------------ */
static inline double rho_of(const or_phys* p, double a) { return a * p->rho_l + (1.0 - a) * p->rho_g; }
static inline double mu_of(const or_phys* p, double a) { return a * p->mu_l + (1.0 - a) * p->mu_g; }

int or_beta(const or_grid* g, const or_phys* p, const double* a, double* bx, double* by,
            double* bz) {
    if (g->per_x || g->per_y) return -1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i)
                bx[U_(g, i, j, k)] = (i == 0 || i == g->nx) ? 0.0
                    : 1.0 / (0.5 * (rho_of(p, a[C_(g, i - 1, j, k)]) + rho_of(p, a[C_(g, i, j, k)])));
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                by[V_(g, i, j, k)] = (j == 0 || j == g->ny) ? 0.0
                    : 1.0 / (0.5 * (rho_of(p, a[C_(g, i, j - 1, k)]) + rho_of(p, a[C_(g, i, j, k)])));
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                bz[W_(g, i, j, k)] =
                    1.0 / (0.5 * (rho_of(p, a[C_(g, i, j, k - 1)]) + rho_of(p, a[C_(g, i, j, k)])));
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pressure operator and Jacobi-preconditioned CG                            */
/* ------------------------------------------------------------------------ */
/* (A P)_c = (1/h^2) sum over the six faces of beta_f (P_c - P_nb); wall
 * faces carry beta = 0. Written with differences so that the residual of a
 * converged solution is not swamped by rounding of P itself. */
static double A_at(const or_grid* g, const double* bx, const double* by, const double* bz,
                   const double* P, int i, int j, int k) {
    double pc = P[C_(g, i, j, k)], s = 0.0;
    if (i > 0) s += bx[U_(g, i, j, k)] * (pc - P[C_(g, i - 1, j, k)]);
    if (i < g->nx - 1) s += bx[U_(g, i + 1, j, k)] * (pc - P[C_(g, i + 1, j, k)]);
    if (j > 0) s += by[V_(g, i, j, k)] * (pc - P[C_(g, i, j - 1, k)]);
    if (j < g->ny - 1) s += by[V_(g, i, j + 1, k)] * (pc - P[C_(g, i, j + 1, k)]);
    s += bz[W_(g, i, j, k)] * (pc - P[C_(g, i, j, k - 1)]);
    s += bz[W_(g, i, j, k + 1)] * (pc - P[C_(g, i, j, k + 1)]);
    return s / (g->h * g->h);
}

int or_apply_A(const or_grid* g, const double* bx, const double* by, const double* bz,
               const double* P, double* AP) {
    if (g->per_x || g->per_y) return -1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) AP[C_(g, i, j, k)] = A_at(g, bx, by, bz, P, i, j, k);
    return 0;
}

static double dot(const or_grid* g, const double* x, const double* y, double* part) {
    const long plane = (long)g->nx * g->ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        double s = 0.0;
        for (long c = k * plane; c < (k + 1) * plane; ++c) s += x[c] * y[c];
        part[k] = s;
    }
    return ordered_sum(part, g->nz);
}

static double mean_of(const or_grid* g, const double* x, double* part) {
    const long plane = (long)g->nx * g->ny;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        double s = 0.0;
        for (long c = k * plane; c < (k + 1) * plane; ++c) s += x[c];
        part[k] = s;
    }
    return ordered_sum(part, g->nz) / (double)ncells(g);
}

int or_solve(const or_grid* g, const double* bx, const double* by, const double* bz,
             const double* b_in, double* P, double rtol, int max_iter, or_report* rep) {
    if (g->per_x || g->per_y) return -1;
    long N = ncells(g);
    const long plane = (long)g->nx * g->ny;
    double* b = (double*)malloc(sizeof(double) * (size_t)N);
    double* r = (double*)malloc(sizeof(double) * (size_t)N);
    double* z = (double*)malloc(sizeof(double) * (size_t)N);
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    double* Dinv = (double*)malloc(sizeof(double) * (size_t)N);
    double* part = (double*)malloc(sizeof(double) * (size_t)g->nz);
    if (!b || !r || !z || !p || !q || !Dinv || !part) return -2;

    /* singular Neumann/periodic operator: the right side must be mean-free */
    double bm = mean_of(g, b_in, part);
    for (long c = 0; c < N; ++c) b[c] = b_in[c] - bm;

    /* Jacobi preconditioner: inverse of the operator diagonal */
    double ih2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double dsum = bx[U_(g, i, j, k)] + bx[U_(g, i + 1, j, k)] + by[V_(g, i, j, k)] +
                              by[V_(g, i, j + 1, k)] + bz[W_(g, i, j, k)] + bz[W_(g, i, j, k + 1)];
                Dinv[C_(g, i, j, k)] = dsum > 0.0 ? 1.0 / (dsum * ih2) : 0.0;
            }

    double bnorm = sqrt(dot(g, b, b, part));
    if (bnorm < 1e-300) bnorm = 1e-300;
    int it = 0, restarts = 0;
    double res0 = 0.0, res = 0.0;
    int converged = 0;
    for (;;) { /* (re)start from the true residual */
        or_apply_A(g, bx, by, bz, P, q);
        for (long c = 0; c < N; ++c) r[c] = b[c] - q[c];
        res = sqrt(dot(g, r, r, part)) / bnorm;
        if (restarts == 0) res0 = res;
        if (res <= rtol) { converged = 1; break; }
        if (it >= max_iter || restarts > 20) break;
        for (long c = 0; c < N; ++c) { z[c] = Dinv[c] * r[c]; p[c] = z[c]; }
        double rz = dot(g, r, z, part);
        int inner_done = 0;
        while (it < max_iter) {
            ++it;
            or_apply_A(g, bx, by, bz, p, q);
            double pq = dot(g, p, q, part);
            if (!(pq > 0.0)) break;
            double al = rz / pq;
#pragma omp parallel for schedule(static)
            for (int k = 0; k < g->nz; ++k)
                for (long c = k * plane; c < (k + 1) * plane; ++c) {
                    P[c] += al * p[c];
                    r[c] -= al * q[c];
                }
            double rr = sqrt(dot(g, r, r, part)) / bnorm;
            if (rr <= rtol) { inner_done = 1; break; }
            for (long c = 0; c < N; ++c) z[c] = Dinv[c] * r[c];
            double rz_new = dot(g, r, z, part);
            double be = rz_new / rz;
            rz = rz_new;
            for (long c = 0; c < N; ++c) p[c] = z[c] + be * p[c];
        }
        ++restarts;
        (void)inner_done;
    }
    double pm = mean_of(g, P, part);
    for (long c = 0; c < N; ++c) P[c] -= pm;
    if (rep) {
        rep->iters = it;
        rep->res0 = res0;
        rep->res = res;
        rep->b_mean = bm;
    }
    free(b); free(r); free(z); free(p); free(q); free(Dinv); free(part);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Momentum predictor (steps 8-10). Velocities are cell-centred (the         */
/* momentum variable) and on faces (the divergence-free advecting field).    */
/* Momentum is convected with the mass fluxes of the geometric VOF sweep,    */
/* sum_k rho_k (phase volume flux), so rho^{n+1} from alpha^{n+1} is exactly */
/* the density these fluxes produce when div u_f = 0 (step 9).               */
/* ------------------------------------------------------------------------ */
/* cell velocity component with no-slip ghosts: every component changes sign
 * across a wall (zero velocity on the wall face) */
static double VC(const or_grid* g, const double* q, int i, int j, int k) {
    double s = 1.0;
    if (i < 0) { i = 0; s = -s; } else if (i >= g->nx) { i = g->nx - 1; s = -s; }
    if (j < 0) { j = 0; s = -s; } else if (j >= g->ny) { j = g->ny - 1; s = -s; }
    return s * q[C_(g, i, j, k)];
}
static double MUC(const or_grid* g, const or_phys* p, const double* a, int i, int j, int k) {
    if (i < 0) i = 0;
    if (i >= g->nx) i = g->nx - 1;
    if (j < 0) j = 0;
    if (j >= g->ny) j = g->ny - 1;
    return mu_of(p, a[C_(g, i, j, k)]);
}

/* Viscous force (component comp) on cell (i,j,k): (1/h) sum over the six
 * faces of the outward traction mu_f (d q_comp/d x_d + d q_d/d x_comp),
 * mu_f the linear face average of the cell viscosities (step 10), normal
 * derivatives from the two cells, tangential ones averaged from the central
 * differences in the two cells. */
static double viscous(const or_grid* g, const or_phys* p, const double* a, const double* const U[3],
                      int comp, int i, int j, int k) {
    const double h = g->h;
    double s = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
            const double sg = side ? 1.0 : -1.0;
            int o[3] = {0, 0, 0};
            o[d] = side ? 1 : -1;
            const int ni = i + o[0], nj = j + o[1], nk = k + o[2];
            const double muf = 0.5 * (MUC(g, p, a, i, j, k) + MUC(g, p, a, ni, nj, nk));
            const double dq = sg * (VC(g, U[comp], ni, nj, nk) - VC(g, U[comp], i, j, k)) / h;
            double dt_ = dq; /* d == comp: the two terms coincide */
            if (d != comp) {
                int e[3] = {0, 0, 0};
                e[comp] = 1;
                const double g1 = (VC(g, U[d], i + e[0], j + e[1], k + e[2]) -
                                   VC(g, U[d], i - e[0], j - e[1], k - e[2])) / (2.0 * h);
                const double g2 = (VC(g, U[d], ni + e[0], nj + e[1], nk + e[2]) -
                                   VC(g, U[d], ni - e[0], nj - e[1], nk - e[2])) / (2.0 * h);
                dt_ = 0.5 * (g1 + g2);
            }
            s += sg * muf * (dq + dt_);
        }
    return s / h;
}

/* Convective momentum change of component q over the step on cell (i,j,k):
 * sum over faces of (outward) M_f q*_f, M_f = rho_l F_f + rho_g (u_f dt/h -
 * F_f) with F_f the liquid volume flux of the VOF sweep (cell volumes);
 * q*_f the donor cell's value (upwind) or the two-cell mean (central). */
static double convection(const or_grid* g, const or_phys* p, const double* q, const double* u,
                         const double* v, const double* w, const double* fx, const double* fy,
                         const double* fz, double dt, int i, int j, int k) {
    double c = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side) {
            int li = i, lj = j, lk = k; /* left cell of the face */
            long f;
            double uf, F;
            if (d == 0) {
                const int fi = i + side;
                if (fi == 0 || fi == g->nx) continue; /* wall: no mass flux */
                li = fi - 1;
                f = U_(g, fi, j, k);
                uf = u[f];
                F = fx[f];
            } else if (d == 1) {
                const int fj = j + side;
                if (fj == 0 || fj == g->ny) continue;
                lj = fj - 1;
                f = V_(g, i, fj, k);
                uf = v[f];
                F = fy[f];
            } else {
                const int fk = k + side;
                lk = fk - 1;
                f = W_(g, i, j, fk);
                uf = w[f];
                F = fz[f];
            }
            int ri = li, rj = lj, rk = lk;
            if (d == 0) ri++; else if (d == 1) rj++; else rk++;
            const double M = p->rho_l * F + p->rho_g * (uf * dt / g->h - F);
            const double qL = q[C_(g, li, lj, lk)], qR = q[C_(g, ri, rj, rk)];
            const double qs = p->conv_scheme == 1 ? (uf > 0.0 ? qL : qR) : 0.5 * (qL + qR);
            c += (side ? 1.0 : -1.0) * M * qs;
        }
    return c;
}

int or_predict(const or_grid* g, const or_phys* p, const double* alpha_n, const double* alpha_np1,
               const double* uc, const double* vc, const double* wc, const double* u,
               const double* v, const double* w, const double* fx, const double* fy,
               const double* fz, double dt, double* uhc, double* vhc, double* whc) {
    if (g->per_x || g->per_y) return -1;
    const double* const U[3] = {uc, vc, wc};
    double* const OUT[3] = {uhc, vhc, whc};
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                const long c = C_(g, i, j, k);
                const double rn = rho_of(p, alpha_n[c]), rn1 = rho_of(p, alpha_np1[c]);
                for (int comp = 0; comp < 3; ++comp) {
                    const double C = convection(g, p, U[comp], u, v, w, fx, fy, fz, dt, i, j, k);
                    const double V = viscous(g, p, alpha_n, U, comp, i, j, k);
                    const double B = comp == 2 ? (rn - p->rho0) * p->g_z + p->dpdz : 0.0;
                    OUT[comp][c] = (rn * U[comp][c] - C + dt * (V + B)) / rn1;
                }
            }
    return 0;
}

/* step 10: face velocities as the linear average of the two cell values */
int or_cell_to_face(const or_grid* g, const double* uc, const double* vc, const double* wc,
                    double* u, double* v, double* w) {
    if (g->per_x || g->per_y) return -1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i)
                u[U_(g, i, j, k)] = (i == 0 || i == g->nx) ? 0.0
                    : 0.5 * (uc[C_(g, i - 1, j, k)] + uc[C_(g, i, j, k)]);
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                v[V_(g, i, j, k)] = (j == 0 || j == g->ny) ? 0.0
                    : 0.5 * (vc[C_(g, i, j - 1, k)] + vc[C_(g, i, j, k)]);
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i)
                w[W_(g, i, j, k)] = 0.5 * (wc[C_(g, i, j, k - 1)] + wc[C_(g, i, j, k)]);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Projection (steps 11-12)                                                  */
/* ------------------------------------------------------------------------ */
int or_rhs(const or_grid* g, const double* bx, const double* by, const double* bz,
           const double* u, const double* v, const double* w, const double* sx,
           const double* sy, const double* sz, double dt, double* b) {
    if (g->per_x || g->per_y) return -1;
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long ulo = U_(g, i, j, k), uhi = U_(g, i + 1, j, k);
                long vlo = V_(g, i, j, k), vhi = V_(g, i, j + 1, k);
                long wlo = W_(g, i, j, k), whi = W_(g, i, j, k + 1);
                /* wall faces carry no flux */
                double ul = i == 0 ? 0.0 : u[ulo], uh = i == g->nx - 1 ? 0.0 : u[uhi];
                double vl = j == 0 ? 0.0 : v[vlo], vh = j == g->ny - 1 ? 0.0 : v[vhi];
                double div_u = (uh - ul + vh - vl + w[whi] - w[wlo]) / h;
                double fl = i == 0 ? 0.0 : bx[ulo] * sx[ulo], fh = i == g->nx - 1 ? 0.0 : bx[uhi] * sx[uhi];
                double gl = j == 0 ? 0.0 : by[vlo] * sy[vlo], gh = j == g->ny - 1 ? 0.0 : by[vhi] * sy[vhi];
                double div_bs = (fh - fl + gh - gl + bz[whi] * sz[whi] - bz[wlo] * sz[wlo]) / h;
                b[C_(g, i, j, k)] = -div_u / dt - div_bs;
            }
    return 0;
}

/* Face acceleration a_f = beta_f ((P_R - P_L)/h - s_f) (zero on walls);
 * u_f -= dt a_f, and each cell component -= dt times the mean of the
 * accelerations on its two faces in that direction (f -> c averaging of
 * step 12). Reports max|div u_f| and max|u_f|. */
int or_correct(const or_grid* g, const double* bx, const double* by, const double* bz,
               const double* P, const double* sx, const double* sy, const double* sz, double dt,
               double* uc, double* vc, double* wc, double* u, double* v, double* w,
               or_report* rep) {
    if (g->per_x || g->per_y) return -1;
    const double h = g->h;
    const long nu = (long)(g->nx + 1) * g->ny * g->nz, nv = (long)g->nx * (g->ny + 1) * g->nz,
               nw = ncells(g);
    double* ax = (double*)calloc((size_t)nu, sizeof(double));
    double* ay = (double*)calloc((size_t)nv, sizeof(double));
    double* az = (double*)calloc((size_t)nw, sizeof(double));
    double* dpart = (double*)calloc((size_t)g->nz, sizeof(double));
    double* upart = (double*)calloc((size_t)g->nz, sizeof(double));
    if (!ax || !ay || !az || !dpart || !upart) return -2;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        for (int j = 0; j < g->ny; ++j)
            for (int i = 1; i < g->nx; ++i) {
                long f = U_(g, i, j, k);
                ax[f] = bx[f] * ((P[C_(g, i, j, k)] - P[C_(g, i - 1, j, k)]) / h - sx[f]);
            }
        for (int j = 1; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long f = V_(g, i, j, k);
                ay[f] = by[f] * ((P[C_(g, i, j, k)] - P[C_(g, i, j - 1, k)]) / h - sy[f]);
            }
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long f = W_(g, i, j, k);
                az[f] = bz[f] * ((P[C_(g, i, j, k)] - P[C_(g, i, j, k - 1)]) / h - sz[f]);
            }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i <= g->nx; ++i) {
                long f = U_(g, i, j, k);
                u[f] = (i == 0 || i == g->nx) ? 0.0 : u[f] - dt * ax[f];
            }
        for (int j = 0; j <= g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long f = V_(g, i, j, k);
                v[f] = (j == 0 || j == g->ny) ? 0.0 : v[f] - dt * ay[f];
            }
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long f = W_(g, i, j, k);
                w[f] = w[f] - dt * az[f];
            }
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long c = C_(g, i, j, k);
                uc[c] -= dt * 0.5 * (ax[U_(g, i, j, k)] + ax[U_(g, i + 1, j, k)]);
                vc[c] -= dt * 0.5 * (ay[V_(g, i, j, k)] + ay[V_(g, i, j + 1, k)]);
                wc[c] -= dt * 0.5 * (az[W_(g, i, j, k)] + az[W_(g, i, j, k + 1)]);
            }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k < g->nz; ++k) {
        double md = 0.0, mu = 0.0;
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double dv = (u[U_(g, i + 1, j, k)] - u[U_(g, i, j, k)] + v[V_(g, i, j + 1, k)] -
                             v[V_(g, i, j, k)] + w[W_(g, i, j, k + 1)] - w[W_(g, i, j, k)]) / h;
                if (fabs(dv) > md) md = fabs(dv);
                double a1 = fabs(u[U_(g, i + 1, j, k)]), a2 = fabs(v[V_(g, i, j + 1, k)]), a3 = fabs(w[W_(g, i, j, k)]);
                if (a1 > mu) mu = a1;
                if (a2 > mu) mu = a2;
                if (a3 > mu) mu = a3;
            }
        dpart[k] = md;
        upart[k] = mu;
    }
    if (rep) {
        double md = 0.0, mu = 0.0;
        for (int k = 0; k < g->nz; ++k) {
            if (dpart[k] > md) md = dpart[k];
            if (upart[k] > mu) mu = upart[k];
        }
        rep->max_div = md;
        rep->max_u = mu;
    }
    free(ax); free(ay); free(az); free(dpart); free(upart);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One time step, Section 2.2 steps 1-12 (with the readings listed above)    */
/* ------------------------------------------------------------------------ */
int or_step(const or_grid* g, const or_phys* p, double* alpha, double* uc, double* vc, double* wc,
            double* u, double* v, double* w, double* P, double dt, long step_index, double rtol,
            int max_iter, or_report* rep) {
    if (g->per_x || g->per_y) return -1;
    long N = ncells(g);
    size_t nu = (size_t)(g->nx + 1) * g->ny * g->nz, nv = (size_t)g->nx * (g->ny + 1) * g->nz,
           nw = (size_t)N;
    double* an = (double*)malloc(sizeof(double) * (size_t)N);
    double* fx = (double*)malloc(sizeof(double) * nu);
    double* fy = (double*)malloc(sizeof(double) * nv);
    double* fz = (double*)malloc(sizeof(double) * nw);
    double* bx = (double*)malloc(sizeof(double) * nu);
    double* by = (double*)malloc(sizeof(double) * nv);
    double* bz = (double*)malloc(sizeof(double) * nw);
    double* sx = (double*)malloc(sizeof(double) * nu);
    double* sy = (double*)malloc(sizeof(double) * nv);
    double* sz = (double*)malloc(sizeof(double) * nw);
    double* hc[3];
    for (int d = 0; d < 3; ++d) hc[d] = (double*)malloc(sizeof(double) * (size_t)N);
    double* kap = (double*)malloc(sizeof(double) * (size_t)N);
    double* b = (double*)malloc(sizeof(double) * (size_t)N);
    if (!an || !fx || !fy || !fz || !bx || !by || !bz || !sx || !sy || !sz || !hc[0] || !hc[1] ||
        !hc[2] || !kap || !b)
        return -2;
    or_report local;
    memset(&local, 0, sizeof(local));

    /* steps 1-2: the level-n state (rho^n, mu^n follow from alpha^n) */
    memcpy(an, alpha, sizeof(double) * (size_t)N);
    /* step 3: advance alpha with the face velocities u_f^n, keeping the
     * liquid volume fluxes for the momentum transport */
    or_advect(g, alpha, u, v, w, dt, step_index, fx, fy, fz, &local);
    /* steps 8-9: cell-centred intermediate velocity (rho^{n+1} from alpha^{n+1}) */
    or_predict(g, p, an, alpha, uc, vc, wc, u, v, w, fx, fy, fz, dt, hc[0], hc[1], hc[2]);
    memcpy(uc, hc[0], sizeof(double) * (size_t)N);
    memcpy(vc, hc[1], sizeof(double) * (size_t)N);
    memcpy(wc, hc[2], sizeof(double) * (size_t)N);
    /* step 10: intermediate face velocities by linear averaging */
    or_cell_to_face(g, uc, vc, wc, u, v, w);
    /* step 4 (beta from rho^{n+1}) and steps 5-7 (curvature, face force) */
    or_beta(g, p, alpha, bx, by, bz);
    or_ssf(g, p, alpha, kap, sx, sy, sz, &local);
    /* step 11: pressure with the surface-tension jump; step 12: correction */
    or_rhs(g, bx, by, bz, u, v, w, sx, sy, sz, dt, b);
    int st = or_solve(g, bx, by, bz, b, P, rtol, max_iter, &local);
    or_correct(g, bx, by, bz, P, sx, sy, sz, dt, uc, vc, wc, u, v, w, &local);
    if (rep) *rep = local;
    free(an); free(fx); free(fy); free(fz); free(bx); free(by); free(bz);
    free(sx); free(sy); free(sz); free(hc[0]); free(hc[1]); free(hc[2]); free(kap); free(b);
    return st;
}
