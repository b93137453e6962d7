/*
 * vof.h -- C ABI of a single-GPU (sm_103a) projection time step for
 * incompressible air-water flow with a volume-of-fluid interface and the
 * sharp-surface-force (SSF) pressure jump, after Kumar & Vanka, "Large Scale
 * GPU Based Simulations of Turbulent Bubbly Flow in a Square Duct",
 * Section 2 (Eqs. 1-7, solution procedure steps 1-12) and Section 4.
 *
 * Grid and layout (all fields FP64, x fastest, caller-owned DEVICE memory,
 * contiguous, no padding):
 *   cells    nx*ny*nz                     index i + nx*(j + ny*k)
 *   u        (nx+1)*ny*nz  x-faces       index i + (nx+1)*(j + ny*k); face i
 *                                        lies between cells i-1 and i
 *   v        nx*(ny+1)*nz  y-faces       index i + nx*(j + (ny+1)*k)
 *   w        nx*ny*nz      z-faces       index i + nx*(j + ny*k); face k lies
 *                                        between cells k-1 and k (periodic)
 * The duct has no-slip walls at x = 0, nx*h and y = 0, ny*h (the wall faces
 * i = 0, nx of u and j = 0, ny of v carry zero velocity and are written as
 * zero by project/step) and is periodic in z (Section 4). alpha is the
 * liquid volume fraction (1 liquid, 0 gas). Pressure P is cell-centred and
 * is the total pressure p + p_tilde of steps 6 and 11 (the surface-tension
 * pressure and the dynamic pressure, obtained from one solve because both
 * elliptic problems share the operator and are linear in their sources).
 *
 * Velocity lives in two places, as in the paper's collocated solver
 * (Section 2, steps 8-12): cell-centred (uc, vc, wc; cell layout), the
 * momentum variable, and on faces (u, v, w), the divergence-free field that
 * advects alpha and carries the mass fluxes.
 *
 * Calls are asynchronous on the context's stream except where a report is
 * requested: then the call synchronises the stream before returning so the
 * report is complete. Errors are return codes; vof_last_error() gives a
 * message. A context is not thread-safe; use one per host thread/stream.
 * There is no CPU fallback: every arithmetic step runs in CUDA kernels.
 */
#ifndef VOF_H
#define VOF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VOF_OK = 0,
    VOF_ERR_ARG = 1,            /* bad size, pointer, flag or value           */
    VOF_ERR_OOM = 2,            /* device allocation failed                   */
    VOF_ERR_CUDA = 3,           /* a CUDA runtime call failed                 */
    VOF_ERR_NOT_CONVERGED = 4,  /* pressure solve hit max_iter (p = last iterate) */
    VOF_ERR_NONFINITE = 5,      /* NaN/Inf in a residual norm                 */
    VOF_ERR_CFL = 6,            /* |u| dt / h > 1 on some face                */
    VOF_ERR_TIMEOUT = 7,        /* a bounded device wait ran out              */
    VOF_ERR_ADMISSION = 8,      /* workspace exceeds the memory budget        */
    VOF_ERR_UNSUPPORTED = 9     /* valid request the library does not support */
} vof_status;

typedef struct {
    int nx, ny, nz;       /* cells; nx, ny >= 2; nz >= 4 and even            */
    double h;             /* uniform spacing (m)                              */
    int periodic_x;       /* 1: x periodic instead of walls (vof_advect only) */
    int periodic_y;       /* 1: y periodic instead of walls (vof_advect only) */
} vof_grid;

enum { VOF_CONV_CENTRAL = 0, VOF_CONV_UPWIND = 1 };
enum { VOF_KAPPA_HEIGHT_FUNCTION = 0, VOF_KAPPA_EXACT = 1 };

typedef struct {
    double rho_l, rho_g;  /* densities (Eq. 4)                                 */
    double mu_l, mu_g;    /* viscosities (Eq. 5)                               */
    double sigma;         /* surface tension coefficient (Eq. 2)               */
    double g_z;           /* gravity along z (negative: downward, Section 4)   */
    double rho0;          /* density whose weight is removed (Section 4)       */
    double dpdz;          /* imposed mean driving force per volume along +z    */
    int conv_scheme;      /* VOF_CONV_*                                        */
    int kappa_mode;       /* VOF_KAPPA_*                                       */
    double kappa_exact;   /* curvature used when kappa_mode == EXACT (1/m)     */
} vof_phys;

/* FP64: flexible CG in FP64 preconditioned by an FP64 V-cycle.
 * MIXED_FP32: FP64 defect correction (residual b - A P and the update of P
 * in FP64) around an inner flexible CG in FP32 preconditioned by an FP32
 * V-cycle. */
enum { VOF_PREC_FP64 = 0, VOF_PREC_MIXED_FP32 = 1 };

typedef struct {
    int precision;        /* VOF_PREC_*: multigrid preconditioner precision   */
    double rtol;          /* stop when ||b - A P||_2 <= rtol ||b||_2          */
    int max_iter;         /* Krylov iteration cap                             */
    int nu_pre, nu_post;  /* red-black Gauss-Seidel sweeps per level (equal)  */
    double mg_omega;      /* scale of the coarse-grid correction, (0, 2];
                             0 selects the default 1                          */
    int coarse_iters;     /* CG iterations cap on the coarsest level; 0 = 400 */
    double coarse_tol;    /* relative residual target there; 0 = default      */
    int mg_interp;        /* VOF_MG_CONSTANT or VOF_MG_TRILINEAR prolongation
                             (restriction is its transpose / 8 in both)       */
    int mg_coarsen;       /* coarse-level coefficients: VOF_COARSEN_FACE_MEAN
                             (mean of the four fine faces a coarse face
                             covers) or VOF_COARSEN_DENSITY_MEAN (density
                             averaged over the eight children, faces then
                             formed by the fine rule 2 / (rho_L + rho_R))    */
    int mg_cycle;         /* VOF_CYCLE_W (default): every level visits its
                             coarser level twice (once when that one is the
                             coarsest, solved exactly); VOF_CYCLE_V: once    */
    int mg_w_depth;       /* W-cycle only: the levels l < mg_w_depth visit
                             their coarser level twice, deeper levels once;
                             0 selects 3 (the tiny levels, launch-latency
                             bound, gain nothing from a second visit)        */
    int graph;            /* on a capturable stream (not the legacy default
                             stream), VOF_GRAPH_AUTO (default): the FP64
                             path captures its V-cycle into a CUDA graph and
                             replays it; the mixed path captures its whole
                             pressure solve, with the inner and refinement
                             loops as conditional WHILE nodes steered by
                             device-side control kernels, and replays it
                             (one launch and one host wait per solve; a
                             graph per right-side/solution pointer pair, two
                             kept); VOF_GRAPH_CYCLE: the V-cycle graph with
                             the loops driven from the host (faster for many
                             contexts running side by side); VOF_GRAPH_OFF:
                             direct launches always. All three give the
                             same iterates.                                */
    int nu_fine;          /* sweeps before and after on the finest level
                             (0: nu_pre, like every other level)             */
    int ssf_solves;       /* 1 (or 0, the default): one solve for the total
                             pressure P = p + p~ with b carrying div(beta s);
                             2: the paper's two solves (steps 6 and 11), p~
                             from div(beta s) and p from div(u_hat)/dt, then
                             P = p + p~ (equal up to the solver tolerance)   */
    int mg_tail;          /* VOF_TAIL_LAUNCHES (default): one launch per
                             smoothing pass, restriction and coarsest solve
                             on every level (replayed from the cycle's CUDA
                             graph); VOF_TAIL_CLUSTER (mixed path with the
                             dense coarsest solve): from the first level of
                             at most 8192 cells down, each visit of the cycle
                             runs as one launch on one thread-block cluster,
                             its operations separated by cluster barriers,
                             with the same arithmetic (equal iterates);
                             VOF_TAIL_GRID: the same from the first level of
                             at most 131072 cells down, each visit one
                             cooperative launch over every SM with its
                             operations separated by grid-wide barriers
                             (bounded waits: VOF_ERR_TIMEOUT if one gives up) */
    int mg_tune;          /* VOF_TUNE_AUTO (default): when the context is
                             created (and when an ensemble sets up its
                             batched solve), the launch shapes of the coarse
                             levels' colour passes (z chunk of a tiled pass,
                             threads of a 1-D block) and of the 1-D
                             restriction from a narrow level are timed on
                             the level's own arrays and the fastest kept;
                             the result is cached per level shape and batch
                             for the process. VOF_TUNE_OFF: the built-in
                             shapes (the request server's contexts always
                             use these: shapes timed for a context alone
                             lose when several share the GPU). The passes
                             are pointwise, so every shape gives the same
                             bits (vof_mg_shape reports the choice). */
} vof_solver;

enum { VOF_COARSEN_FACE_MEAN = 0, VOF_COARSEN_DENSITY_MEAN = 1 };
enum { VOF_CYCLE_W = 0, VOF_CYCLE_V = 1 };
enum { VOF_GRAPH_AUTO = 0, VOF_GRAPH_OFF = 1, VOF_GRAPH_CYCLE = 2 };
enum { VOF_TAIL_LAUNCHES = 0, VOF_TAIL_CLUSTER = 1, VOF_TAIL_GRID = 2 };
enum { VOF_TUNE_AUTO = 0, VOF_TUNE_OFF = 1 };

enum { VOF_MG_CONSTANT = 0, VOF_MG_TRILINEAR = 1 };

typedef struct {
    int iters;                    /* Krylov iterations of the last solve (mixed:
                                     inner FP32 iterations summed)              */
    int refinements;              /* mixed: FP64 defect-correction steps        */
    double res0, res;             /* initial / final relative residual          */
    double b_mean;                /* mean removed from the right side           */
    double vol_before, vol_after; /* liquid volume sum(alpha) h^3 (m^3)         */
    double vol_clipped;           /* volume added by clipping alpha to [0,1]    */
    double max_div;               /* max |div u| after the projection (1/s)     */
    double max_u;                 /* max |face velocity| after projection (m/s) */
    long long hf_fallbacks;       /* faces whose curvature needed the fallback  */
    float ms[8];                  /* advect, ssf, predict, rhs, solve, project,
                                     other, total (ms; filled when timing is on) */
} vof_report;

typedef struct vof_ctx vof_ctx;

/* Device memory a context for this grid/solver needs (bytes), without
 * allocating anything. Returns VOF_ERR_ARG for an invalid grid. */
vof_status vof_workspace_bytes(const vof_grid* grid, const vof_solver* solver, size_t* bytes);

/* Create a context on the current CUDA device: validates the grid, physics
 * and solver settings and allocates the whole workspace once (multigrid
 * hierarchy, Krylov vectors, scratch). budget_bytes > 0 caps that workspace
 * (VOF_ERR_ADMISSION if exceeded); 0 means no cap. stream is a cudaStream_t
 * (NULL = legacy default stream). On failure *out is NULL. */
vof_status vof_create(const vof_grid* grid, const vof_phys* phys, const vof_solver* solver,
                      size_t budget_bytes, void* stream, vof_ctx** out);
vof_status vof_destroy(vof_ctx* ctx);
const char* vof_last_error(const vof_ctx* ctx);

/* Advance alpha in place by one time step of dt with the face velocities
 * (u, v, w) (Eq. 3): PLIC reconstruction with the normal from the smoothed
 * volume fraction (Section 2, Rudman), plane constants in FP64, and
 * geometric donor-slab fluxes in three direction-split sweeps (x, y, z when
 * step_index is even, z, y, x when odd; the "second-order operator split"
 * of Section 2.1), the divergence term weighted by [alpha^n > 1/2] so the
 * liquid volume is conserved to round-off when div u = 0 (abstract:
 * absolute mass conservation). Wall-face values of u, v are ignored.
 * fx, fy, fz (optional, NULL to skip; face layouts as u, v, w): the signed
 * liquid volume that crossed each face in its sweep, in cell volumes -- the
 * mass fluxes vof_predict needs. VOF_ERR_CFL if some |u| dt/h > 1. report
 * (optional) gets the volumes. */
vof_status vof_advect(vof_ctx* ctx, double* alpha, const double* u, const double* v,
                      const double* w, double dt, long long step_index, double* fx, double* fy,
                      double* fz, vof_report* report);

/* Interface curvature and the sharp surface force on faces (Eq. 6, steps
 * 5-7): kappa per cell from height functions (Section 2, Cummins et al.;
 * 0 where no valid column exists) or kappa_exact, and
 *   s_f = sigma * kappa_f * (G_R - G_L) / h,  G = [alpha < 1/2],
 * with kappa_f the mean of the valid neighbouring cell values. Outputs
 * kappa (cells) and sx, sy, sz (face layouts as u, v, w; zero on walls). */
vof_status ssf_force(vof_ctx* ctx, const double* alpha, double* kappa, double* sx, double* sy,
                     double* sz);

/* Solve the variable-coefficient pressure equation (Eq. 7, steps 6/11)
 *   (A P)_c = (1/h^2) sum_f beta_f (P_c - P_nb) = b_c,
 *   beta_f = 2 / (rho_L + rho_R),  rho = alpha rho_l + (1 - alpha) rho_g,
 * with geometric-multigrid-preconditioned flexible CG. mean(b) is removed
 * (singular operator: walls and periodic z) and reported; p is the initial
 * guess on entry and the mean-free solution on exit. VOF_ERR_NOT_CONVERGED
 * leaves the last iterate in p. */
vof_status pressure_solve(vof_ctx* ctx, const double* alpha, const double* b, double* p,
                          vof_report* report);

/* y = A x with beta from alpha (the operator of pressure_solve). */
vof_status vof_apply_operator(vof_ctx* ctx, const double* alpha, const double* x, double* y);

/* Largest total face count (x + y + z faces) vof_apply_operator_noalloc
 * accepts: its fixed scratch holds this many doubles (24 MiB). */
#define VOF_NOALLOC_MAX_FACES (3u << 20)

/* y = A x as vof_apply_operator computes it (the same kernels, so the same
 * bits), but with no context and no device allocation at all. The paper has
 * no counterpart: it exists for callers that cannot call cudaMalloc -- hosts
 * that reserve all device memory up front in their own arena, where a
 * cudaMalloc would fail or escape their accounting, and latency-critical
 * loops where an allocation could synchronise the device. The face
 * coefficients beta it builds from alpha go into one fixed device array
 * inside the library (24 MiB, held by every GPU that loads the library
 * until the process exits), so
 *  - grids with more than VOF_NOALLOC_MAX_FACES faces in total are
 *    rejected with VOF_ERR_ADMISSION before anything is launched; other
 *    grids and properties are checked as vof_create checks them
 *    (VOF_ERR_ARG);
 *  - every call shares that array and overwrites all of it that it reads,
 *    so nothing needs clearing between calls, but calls whose kernels
 *    overlap on the GPU (different streams, or different host threads on
 *    one device) race on it: serialise them;
 *  - the first call in each CUDA context (each device's primary context,
 *    and again after cudaDeviceReset) looks up the array's device address
 *    (cudaGetSymbolAddress, which may load the library's module), so make
 *    that first call before any stream capture in that context.
 * alpha, x, y: device arrays in the cell layout; stream: cudaStream_t (NULL
 * = legacy default stream); the call is asynchronous on it. Walls only
 * (VOF_ERR_UNSUPPORTED for periodic x or y). */
vof_status vof_apply_operator_noalloc(const vof_grid* grid, const vof_phys* phys,
                                      const double* alpha, const double* x, double* y,
                                      void* stream);

/* Momentum predictor (Eq. 2; steps 8-10). On entry (uc, vc, wc) hold the
 * cell velocity u^n and (u, v, w) the face velocity that advected alpha
 * from alpha_n to alpha_np1 with liquid face fluxes (fx, fy, fz) from
 * vof_advect. On exit (uc, vc, wc) hold the intermediate cell velocity
 *   u_hat = [rho^n u^n - sum_f M_f q*_f + dt (V + B)] / rho^{n+1},
 *   M_f = rho_l F_f + rho_g (u_f dt/h - F_f)   (mass moved by the sweep),
 * q*_f the donor cell's velocity (upwind) or the two-cell mean (central),
 * V the explicit full-stress viscous force, B = (rho^n - rho0) g_z + dpdz on
 * the z-component (Section 4); and (u, v, w) hold u_hat_f, the mean of the
 * two cells (step 10), zero on walls. */
vof_status vof_predict(vof_ctx* ctx, const double* alpha_n, const double* alpha_np1, double* uc,
                       double* vc, double* wc, double* u, double* v, double* w, const double* fx,
                       const double* fy, const double* fz, double dt);

/* Projection (steps 11-12): b = -div(u_hat_f)/dt - div(beta s), solve
 * A P = b (p: initial guess in, solution out), then with the face
 * acceleration a_f = beta_f ((P_R - P_L)/h - s_f):
 *   u_f = u_hat_f - dt a_f,   u_c = u_hat_c - dt (a_f- + a_f+)/2
 * (each cell component takes the mean of its two faces in that direction).
 * (uc, vc, wc) and (u, v, w) are updated in place. report gets iterations,
 * residuals, max|div u_f| and max|u_f|. */
vof_status project(vof_ctx* ctx, const double* alpha, double* uc, double* vc, double* wc, double* u,
                   double* v, double* w, double* p, const double* sx, const double* sy,
                   const double* sz, double dt, vof_report* report);

/* One whole time step (steps 1-12): vof_advect with the face velocities,
 * vof_predict, ssf_force on alpha^{n+1}, project. All arguments are updated
 * in place.
 * glibc also exports a symbol named step (its legacy <regexp.h> matcher).
 * The library is linked -Bsymbolic so its own calls never reach glibc's,
 * and a handle from dlopen finds this one; a program that links the
 * library directly and whose link order puts libc first should call
 * vof_step, the same function under an unambiguous name. */
vof_status step(vof_ctx* ctx, double* alpha, double* uc, double* vc, double* wc, double* u,
                double* v, double* w, double* p, double dt, long long step_index,
                vof_report* report);
vof_status vof_step(vof_ctx* ctx, double* alpha, double* uc, double* vc, double* wc, double* u,
                    double* v, double* w, double* p, double dt, long long step_index,
                    vof_report* report);

/* One time step on a state held in HOST memory: the same step as step(),
 * with the eight arrays (same order, sizes and layouts) in host memory.
 * The context keeps a device copy of the state, allocated by the first call
 * (8 fields, in addition to vof_workspace_bytes; VOF_ERR_OOM if the device
 * has no room). Each call copies the state in on a stream of its own, alpha,
 * u, v and w first (the CFL check and the advection read them) and the cell
 * velocities and p while the advection, beta and the face force run; it
 * copies each field out, on a second stream, as soon as the step has
 * finished writing it: alpha after the advection, p after the solve, the
 * velocities after the projection. Page-locked host arrays (cudaHostAlloc,
 * pinned tensors) let the copies overlap the kernels; pageable ones work,
 * with copies staged by the CUDA runtime.
 * Ordering. The copies in start after all work already on the context
 * stream and, field by field, after the previous call's copy out of the
 * same field. So consecutive calls on the same arrays form a time loop in
 * which a call's copies in overlap the previous call's copies out (the two
 * directions of the bus at once).
 * Completion. With report != NULL the call returns when the step and all
 * its copies have finished: the host arrays hold the new state. With
 * report == NULL the copies out may still run when the call returns and the
 * context stream does not wait for them; vof_host_join orders them before
 * later work on the context stream, so that synchronising the stream after
 * it leaves the host arrays complete. Until then the arrays must stay
 * valid and untouched. Errors as for step(); after an error other than
 * VOF_ERR_NOT_CONVERGED the host arrays are unspecified. */
vof_status vof_step_host(vof_ctx* ctx, double* alpha, double* uc, double* vc, double* wc,
                         double* u, double* v, double* w, double* p, double dt,
                         long long step_index, vof_report* report);

/* Makes the context stream wait for every copy of earlier vof_step_host
 * calls (no-op if there were none); returns at once. */
vof_status vof_host_join(vof_ctx* ctx);

/* Diagnostic of the failure path of the bounded device waits: one block
 * waits, with the same bounded wait as the staged sweep, on a shared-memory
 * barrier that nothing completes (no copy is in flight). The limit runs
 * out, the block sets the context's device error flag, and the call returns
 * VOF_ERR_TIMEOUT, as a solve does when a staged plane never arrives. The
 * flag is cleared again, so the context stays usable. Synchronous. */
vof_status vof_diag_wait_timeout(vof_ctx* ctx);

/* Number of CUDA kernels this context has launched since creation (the
 * launch-shape timing of solver->mg_tune included). */
vof_status vof_launch_count(const vof_ctx* ctx, long long* n);

/* Launch shape of multigrid level `level`'s colour passes (solver->mg_tune):
 * shape[0] the z planes per thread of a tiled pass (0 when the level runs
 * 1-D blocks), shape[1] the threads of a 1-D block of the passes (0 when
 * tiled), shape[2] the threads of a 1-D block of the restriction from this
 * level (0 when that restriction is tiled), shape[3] 1 when the shape was
 * chosen by timing, 0 when built in. VOF_ERR_ARG for a null argument or a
 * level that runs no colour passes through these kernels (the finest level,
 * the coarsest, a level with an odd nx). */
vof_status vof_mg_shape(const vof_ctx* ctx, int level, int shape[4]);
/* Sets that shape: shape[0..2] as vof_mg_shape reports them, nonzero
 * exactly where the level uses a value (z planes per thread in [1, nz];
 * block threads a multiple of 32 in [32, 1024]); the shape then counts as
 * built in. It applies to the launches made, and the graphs captured, after
 * the call: set it before the first solve. Any valid shape gives the same
 * bits. VOF_ERR_ARG for a bad level or value, nothing changed. */
vof_status vof_mg_set_shape(vof_ctx* ctx, int level, const int shape[3]);

/* Per-phase CUDA-event timing inside the calls (off by default). When on,
 * kernel classes are bracketed by events on the context stream and the
 * accumulated device time and launch counts are returned by
 * vof_kernel_times (then reset). Classes: "advect", "ssf", "predict", "rhs",
 * "smooth_l0" (fine-grid red-black half-sweeps), "smooth" (coarser levels),
 * "residual_l0" (fine-grid operator applications in the Krylov loop),
 * "restrict_l0", "restrict", "prolong_l0", "prolong", "coarse", "krylov"
 * (fine-grid vector updates), "project"; n = number of classes written
 * (<= cap). */
vof_status vof_set_timing(vof_ctx* ctx, int on);
vof_status vof_kernel_times(vof_ctx* ctx, const char** names, double* ms, long long* launches,
                            int cap, int* n);

/* ---- request server: continuous batching of independent cases ----------
 * The paper has no serving layer; this serves ensembles of independent duct
 * cases (time steps or pressure solves on grids of their own) on one GPU.
 * Requests queue in arrival order; the head request is admitted as soon as
 * one of max_concurrent worker slots is free and its device memory (fields
 * plus context workspace, see vof_workspace_bytes) fits in what is left of
 * budget_bytes. Each admitted request runs on its worker's own CUDA stream,
 * so requests overlap on the device; a result does not depend on what else
 * was running. Host arrays of a request are read when it starts and
 * overwritten with the results when it finishes; they must stay valid until
 * vof_wait/vof_poll report it finished. A request's context exists for that
 * request only, so it launches its kernels directly (solver.graph is taken
 * as VOF_GRAPH_OFF). */
typedef struct vof_server vof_server;

enum { VOF_REQ_STEP = 0, VOF_REQ_SOLVE = 1 };

typedef struct {
    int kind;               /* VOF_REQ_STEP: n_steps calls of step();
                               VOF_REQ_SOLVE: one pressure_solve()           */
    vof_grid grid;
    vof_phys phys;
    vof_solver solver;
    int n_steps;            /* STEP: number of time steps (>= 1)             */
    double dt;              /* STEP: time step                               */
    long long step0;        /* STEP: index of the first step (split order)   */
    double *alpha, *uc, *vc, *wc, *u, *v, *w, *p;  /* HOST arrays, layouts as
                               in step(); SOLVE uses alpha (read), p (guess in,
                               solution out) and b                            */
    const double* b;        /* SOLVE: right side (host)                       */
} vof_request;

typedef struct {
    int status;             /* vof_status of the request; -1 until finished  */
    int state;              /* 0 queued, 1 running, 2 finished               */
    double t_submit, t_admit, t_finish;  /* seconds since server creation    */
    vof_report report;      /* of the solve / of the last step               */
} vof_result;

/* budget_bytes > 0: device memory the admitted requests may hold together;
 * max_concurrent in [1, 64]: worker slots (CUDA streams). Uses the current
 * device, and raises the release threshold of that device's default memory
 * pool (the one cudaMallocAsync draws from) to budget_bytes so that memory
 * freed by a finished request is reused by the next one. */
vof_status vof_server_create(size_t budget_bytes, int max_concurrent, vof_server** out);
/* VOF_ERR_ADMISSION if the request alone exceeds the budget; VOF_ERR_ARG for
 * invalid requests. *id identifies the request. */
vof_status vof_submit(vof_server* server, const vof_request* request, unsigned long long* id);
vof_status vof_poll(vof_server* server, unsigned long long id, vof_result* result);
/* Blocks until the request has finished. */
vof_status vof_wait(vof_server* server, unsigned long long id, vof_result* result);
/* Finishes every queued request, then frees the server. */
vof_status vof_server_destroy(vof_server* server);

/* ---- ensemble of independent ducts ---------------------------------------
 * The paper has no ensemble mode; this advances n_cases independent cases of
 * one grid size by one time step per call, fields resident on the device.
 * Each case has its own context (workspace as vof_create); cases are dealt
 * round-robin to n_streams worker threads, each with its own CUDA stream, so
 * their kernels overlap on the GPU. A case's result is bitwise that of the
 * same case stepped alone by step(). Uses the current device. With
 * solver->graph VOF_GRAPH_AUTO the cases run as VOF_GRAPH_CYCLE (their
 * solves' loops on the host), which is faster for many cases side by side. */
typedef struct vof_ensemble vof_ensemble;

/* phys: n_phys = 1 (shared) or n_cases entries (per case, e.g. rho0).
 * n_streams in [1, 64]. */
vof_status vof_ensemble_create(const vof_grid* grid, const vof_phys* phys, int n_phys,
                               const vof_solver* solver, int n_cases, int n_streams,
                               vof_ensemble** out);
/* fields: 8 * n_cases DEVICE pointers, case c at [8c .. 8c+7] in the order
 * alpha, uc, vc, wc, u, v, w, p (layouts as in step()); dt: n_cases time
 * steps (host array). Blocks until every case has finished its step.
 * status (n_cases, may be NULL) receives each case's status, reports
 * (n_cases, may be NULL) each case's report; the return value is the first
 * non-OK status, else VOF_OK. */
vof_status vof_ensemble_step(vof_ensemble* ensemble, double* const* fields, const double* dt,
                             long long step_index, vof_status* status, vof_report* reports);
vof_status vof_ensemble_destroy(vof_ensemble* ensemble);

/* How an ensemble runs its cases.
 *  VOF_ENSEMBLE_BATCHED: the pressure solves of all cases run as one batched
 *    solve (Eq. 7 for every case at once): the cases' workspaces are carved
 *    from one device arena at a fixed stride, and every multigrid operation
 *    of a level, every Krylov update and every reduction is one launch for
 *    all cases, with per-case sums and per-case convergence (a case whose
 *    loop has ended is switched off, its blocks return at once); the V-cycle
 *    of all cases replays from one CUDA graph. The parts of the step before
 *    and after the solve run per case on the worker streams. Each case's
 *    kernels, block sums and decisions are those of its solo solve, so its
 *    result is bitwise that of the case stepped alone. Needs the mixed
 *    precision with the density-formed finest level (nx a multiple of 8),
 *    constant prolongation, face-mean coarsening, a dense coarsest level, an
 *    even number of finest-level sweeps, the single combined solve and no
 *    cluster tail; otherwise VOF_ERR_UNSUPPORTED.
 *    With solver->graph VOF_GRAPH_AUTO the whole batched step is one CUDA
 *    graph launch: the CFL test of every case (one kernel and a device-side
 *    test), then, under a conditional IF node the test opens, every case's
 *    step up to its solve (the cases' branches side by side), the batched
 *    solve with its two loops as conditional WHILE nodes whose per-case
 *    decisions are taken on the device, and every case's correction. From
 *    8 cases up the cases run in min(4, n_cases / 4) groups of consecutive
 *    cases, each with its own batched solve; a group's step up to its solve
 *    starts when the group before has finished its own, and so runs beside
 *    that group's solve. The
 *    graph is captured at the first step and again whenever the field
 *    pointers, the time steps or the parity of step_index change. A step
 *    whose CFL test fails in any case runs again the host-driven way
 *    (nothing of it was launched), which reports each case's status. In the
 *    graph, a case whose solve fails (non-finite, or a bounded wait gave up)
 *    still has its correction applied from the failed pressure; its status
 *    reports the failure. VOF_GRAPH_CYCLE keeps the loops on the host.
 *  VOF_ENSEMBLE_STREAMS: every case steps through its own context on the
 *    worker streams, overlapping on the GPU.
 *  VOF_ENSEMBLE_AUTO: batched where the solver allows it, else streams
 *    (vof_ensemble_create). */
#define VOF_ENSEMBLE_AUTO 0
#define VOF_ENSEMBLE_STREAMS 1
#define VOF_ENSEMBLE_BATCHED 2
vof_status vof_ensemble_create_mode(const vof_grid* grid, const vof_phys* phys, int n_phys,
                                    const vof_solver* solver, int n_cases, int n_streams,
                                    int mode, vof_ensemble** out);
/* *batched = 1 when the ensemble runs its solves batched, else 0. */
vof_status vof_ensemble_batched(const vof_ensemble* ensemble, int* batched);
/* Kernels launched by the ensemble so far (every case, a batched launch
 * counted once). */
vof_status vof_ensemble_launch_count(const vof_ensemble* ensemble, long long* n);
/* Time (ms) the steps so far spent in their three parts. Host-driven steps
 * (host wall time): ms[0] the parts before the solves (the whole step for a
 * streams ensemble), ms[1] the batched solve, ms[2] the parts after it.
 * Steps run as one graph launch (the device's global timer; the groups'
 * parts overlap): ms[0] from the CFL test to the end of the first group's
 * part before its solve, ms[1] from there to the end of the last group's
 * solve, ms[2] the rest. */
vof_status vof_ensemble_phase_ms(const vof_ensemble* ensemble, double* ms);
/* Steps so far that ran as one graph launch. */
vof_status vof_ensemble_graph_steps(const vof_ensemble* ensemble, long long* n);
/* vof_mg_shape of the batched solve's levels (the launches that cover the
 * first group of cases, or every case when the steps are host-driven);
 * VOF_ERR_UNSUPPORTED for an ensemble without batched solves. */
vof_status vof_ensemble_mg_shape(const vof_ensemble* ensemble, int level, int shape[4]);

/* ---- duct statistics ------------------------------------------------------
 * Running sums for the profiles of Section 4 (averages over the streamwise
 * direction z and over time, mixture and liquid phase). For every column
 * (i, j) of the cross-section, over all z and all samples, the FP64 sums of
 *   q = 0..9:   phi = 1 - alpha, u, v, w, uu, vv, ww, uv, uw, vw
 *   q = 10..19: alpha, and alpha times each of u, v, w, uu, vv, ww, uv, uw, vw
 * (u, v, w the cell-centred velocities). Mixture means are sums / (samples *
 * nz); liquid means are the alpha-weighted sums / sum of alpha. Each column
 * is summed by one thread in z order, so the sums are deterministic. Uses
 * the current device. */
#define VOF_NSTAT 20
typedef struct vof_stats vof_stats;

vof_status vof_stats_create(const vof_grid* grid, vof_stats** out);
/* One sample: DEVICE fields (cell layout) of one state, on the given stream
 * (a cudaStream_t; NULL for the legacy default stream). */
vof_status vof_stats_accumulate(vof_stats* stats, const double* alpha, const double* uc,
                                const double* vc, const double* wc, void* stream);
/* Waits for the device, then copies the sums to sums (host, VOF_NSTAT x ny x
 * nx, q slowest) and the sample count. */
vof_status vof_stats_read(vof_stats* stats, double* sums, long long* samples);
vof_status vof_stats_reset(vof_stats* stats);
vof_status vof_stats_destroy(vof_stats* stats);

#ifdef __cplusplus
}
#endif
#endif
