/*
 * vof_oracle.h -- plain FP64 CPU oracle for one projection time step of the
 * air-water VOF / sharp-surface-force solver of Kumar & Vanka,
 * "Large Scale GPU Based Simulations of Turbulent Bubbly Flow in a Square
 * Duct" (Section 2: Eqs. 1-7 and the twelve-step solution procedure).
 *
 * TEST INFRASTRUCTURE. This file and vof_oracle.c exist only to check the
 * CUDA library against the paper. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may link or call it; the library
 * never does. It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (the same physical discretisation as the CUDA library, written
 * independently):
 *   cells      nx*ny*nz, x fastest: c = i + nx*(j + ny*k); spacing h.
 *   u faces    (nx+1)*ny*nz, face (i,j,k) sits at x = i*h between cells
 *              i-1 and i; index i + (nx+1)*(j + ny*k).
 *   v faces    nx*(ny+1)*nz, face (i,j,k) at y = j*h; index i + nx*(j + (ny+1)*k).
 *   w faces    nx*ny*nz, face (i,j,k) at z = k*h between cells k-1 and k
 *              (periodic in z); index i + nx*(j + ny*k).
 *   x and y are no-slip walls (faces 0 and n hold zero normal velocity)
 *   unless per_x / per_y is set; per_x / per_y are honoured by the VOF
 *   advection only (translation tests). z is always periodic.
 *   alpha is the liquid volume fraction (1 = liquid, 0 = gas).
 */
#ifndef VOF_ORACLE_H
#define VOF_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;
    double h;
    int per_x, per_y;
} or_grid;

typedef struct {
    double rho_l, rho_g, mu_l, mu_g, sigma;
    double g_z;       /* gravity along z (negative = downward) */
    double rho0;      /* reference density removed with the hydrostatic part */
    double dpdz;      /* imposed mean driving force per volume along +z */
    int conv_scheme;  /* 0 = central, 1 = first-order upwind */
    int kappa_mode;   /* 0 = height function, 1 = exact (kappa_exact) */
    double kappa_exact;
} or_phys;

typedef struct {
    int iters;
    double res0, res, b_mean;
    double vol_before, vol_after, vol_clipped;
    double max_div, max_u;
    long hf_fallbacks;
} or_report;

/* Interface threshold: cells with eps < alpha < 1-eps carry a plane. */
#define OR_EPS 1e-12

/* --- PLIC geometry (Section 2.1, interface as an oblique plane) --------- */
/* Volume of {xi in [0,1]^3 : m.xi <= a}. Any signs of m. */
double or_plane_volume(const double m[3], double a);
/* Plane constant a with or_plane_volume(m, a) = alpha, by bisection. */
double or_plane_constant(const double m[3], double alpha);
/* Unnormalised interface normal -(grad of smoothed alpha), cell units. */
void or_normal(const or_grid* g, const double* alpha, int i, int j, int k, double n[3]);
/* Height-function direction chosen from the normal (0=x,1=y,2=z). */
int or_hf_direction(const double n[3]);

/* --- VOF advection (Eq. 3; geometric split fluxes) ----------------------- */
/* fx, fy, fz (optional, may be NULL): signed liquid volume crossing each
 * face during its sweep, in cell volumes, face layouts as u, v, w. */
int or_advect(const or_grid* g, double* alpha, const double* u, const double* v,
              const double* w, double dt, long step_index, double* fx, double* fy, double* fz,
              or_report* rep);

/* --- curvature and sharp surface force (Eqs. 6-7; steps 5-7) ------------ */
/* kappa per cell (0 where not computed), valid flag per cell (may be NULL). */
int or_curvature(const or_grid* g, const double* alpha, double* kappa,
                 unsigned char* valid);
int or_ssf(const or_grid* g, const or_phys* p, const double* alpha,
           double* kappa, double* sx, double* sy, double* sz, or_report* rep);

/* --- mixture properties (Eqs. 4-5; step 10 linear face averaging) -------- */
int or_beta(const or_grid* g, const or_phys* p, const double* alpha,
            double* bx, double* by, double* bz);

/* --- Poisson operator and solve (Eq. 7; steps 6 and 11) ------------------ */
/* (A P)_c = (1/h^2) sum_f beta_f (P_c - P_nb). */
int or_apply_A(const or_grid* g, const double* bx, const double* by,
               const double* bz, const double* P, double* AP);
/* Removes mean(b), solves A P = b by Jacobi-preconditioned CG to
 * ||b - A P||_2 <= rtol ||b||_2 starting from P, then sets mean(P) = 0. */
int or_solve(const or_grid* g, const double* bx, const double* by,
             const double* bz, const double* b, double* P, double rtol,
             int max_iter, or_report* rep);

/* --- momentum predictor (steps 8-10) ------------------------------------- */
/* Cell-centred u_hat = [rho^n u^n - C + dt (V + B)] / rho^{n+1}, C the
 * convective momentum change with the VOF mass fluxes (fluxes from
 * or_advect with the face velocities u, v, w). */
int or_predict(const or_grid* g, const or_phys* p, const double* alpha_n,
               const double* alpha_np1, const double* uc, const double* vc,
               const double* wc, const double* u, const double* v, const double* w,
               const double* fx, const double* fy, const double* fz, double dt,
               double* uhc, double* vhc, double* whc);
/* Face values as the mean of the two cells (zero on walls). */
int or_cell_to_face(const or_grid* g, const double* uc, const double* vc,
                    const double* wc, double* u, double* v, double* w);

/* --- projection (steps 11-12) -------------------------------------------- */
/* b = -div(u_hat_f)/dt - div(beta s). */
int or_rhs(const or_grid* g, const double* bx, const double* by, const double* bz,
           const double* u, const double* v, const double* w, const double* sx,
           const double* sy, const double* sz, double dt, double* b);
/* a_f = beta_f ((P_R - P_L)/h - s_f); u_f -= dt a_f; cells -= dt times the
 * mean of their two face accelerations. Reports max|div u_f|, max|u_f|. */
int or_correct(const or_grid* g, const double* bx, const double* by,
               const double* bz, const double* P, const double* sx,
               const double* sy, const double* sz, double dt, double* uc,
               double* vc, double* wc, double* u, double* v, double* w,
               or_report* rep);

/* --- one whole time step (steps 1-12) ------------------------------------ */
int or_step(const or_grid* g, const or_phys* p, double* alpha, double* uc, double* vc,
            double* wc, double* u, double* v, double* w, double* P, double dt,
            long step_index, double rtol, int max_iter, or_report* rep);

/* Threads used by the OpenMP loops (for the CPU-baseline report), and a
 * cap on them for later calls (n <= 0: unchanged). */
int or_num_threads(void);
void or_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
