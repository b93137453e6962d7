// C ABI of the projection step (include/vof.h): context lifetime, argument
// validation, the workspace, and the five entry points of the time step.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>

#include "vof_internal.cuh"

namespace {

constexpr int P_A = 20, P_B = 21, P_C = 22;  // scratch partial slots

struct Sizes {
    size_t n, nu, nv, nw;
};

Sizes sizes_of(const vof_grid* g) {
    Sizes s;
    s.n = (size_t)g->nx * g->ny * g->nz;
    s.nu = (size_t)(g->nx + 1) * g->ny * g->nz;
    s.nv = (size_t)g->nx * (g->ny + 1) * g->nz;
    s.nw = s.n;
    return s;
}

vof_status alloc(vof_ctx* c, void** p, size_t bytes) {
    *p = dev_alloc(c, bytes);
    if (!*p) return set_err(c, VOF_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes failed");
    return VOF_OK;
}

void flush_timers(vof_ctx* c) {
    if (c->ev_marks.empty()) return;
    cudaStreamSynchronize(c->st);
    for (auto& m : c->ev_marks) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev_pool[m.second.first], c->ev_pool[m.second.second]);
        c->t_ms[m.first] += ms;
        c->t_n[m.first] += 1;
    }
    c->ev_marks.clear();
}

vof_status check_ctx(vof_ctx* c) {
    if (!c) return VOF_ERR_ARG;
    c->err.clear();
    return VOF_OK;
}

#define REQUIRE_PTR(c, p)                                                 \
    do {                                                                  \
        if (!(p)) return set_err((c), VOF_ERR_ARG, #p " is NULL");        \
    } while (0)

vof_status walls_only(vof_ctx* c, const char* who) {
    if (c->g.periodic_x || c->g.periodic_y)
        return set_err(c, VOF_ERR_UNSUPPORTED,
                       std::string(who) + " needs wall boundaries in x and y");
    return VOF_OK;
}

vof_status cfl_check(vof_ctx* c, const double* u, const double* v, const double* w, double dt) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(c, VOF_ERR_ARG, "dt must be positive");
    launch_cfl(c, u, v, w, dt, P_A);
    readback(c);
    const double cfl = c->hbuf[S_CFL] * dt / c->g.h;
    if (!std::isfinite(cfl)) return set_err(c, VOF_ERR_NONFINITE, "non-finite velocity");
    if (cfl > 1.0)
        return set_err(c, VOF_ERR_CFL, "Courant number " + std::to_string(cfl) + " exceeds 1");
    return VOF_OK;
}

// three direction-split sweeps; alpha in place (ping-pong through a1, a2);
// the liquid flux of every face is left in flux[dir]
void advect_impl(vof_ctx* c, double* alpha, const double* u, const double* v, const double* w,
                 double dt, long long step_index, double* const flux[3]) {
    const double h3 = c->g.h * c->g.h * c->g.h;
    int m = timer_begin(c, T_ADVECT);
    launch_vof_mask_volume(c, alpha, P_A);
    timer_end(c, T_ADVECT, m);
    finalize_sum(c, P_A, c->Lc.nblocks, S_VOL0, h3);
    const double* vel[3] = {u, v, w};
    const double* src = alpha;
    for (int s = 0; s < 3; ++s) {
        const int dir = (step_index % 2 == 0) ? s : 2 - s;
        double* dst = s == 2 ? alpha : (s == 0 ? c->a1 : c->a2);
        launch_reconstruct(c, src);
        launch_face_flux(c, dir, src, vel[dir], dt, flux[dir]);
        launch_vof_update(c, dir, src, dst, vel[dir], flux[dir], dt, P_B);
        finalize_sum(c, P_B, c->Lc.nblocks, S_CLIP0 + s, h3);
        src = dst;
    }
    launch_volume(c, alpha, P_A);
    finalize_sum(c, P_A, c->Lc.nblocks, S_VOL1, h3);
}

void fill_vof_report(vof_ctx* c, vof_report* r) {
    r->vol_before = c->hbuf[S_VOL0];
    r->vol_after = c->hbuf[S_VOL1];
    r->vol_clipped = c->hbuf[S_CLIP0] + c->hbuf[S_CLIP1] + c->hbuf[S_CLIP2];
}

void ssf_impl(vof_ctx* c, const double* alpha, double* kappa, double* sx, double* sy, double* sz) {
    launch_curvature(c, alpha, kappa, c->valid);
    launch_ssf_faces(c, alpha, kappa, c->valid, sx, sy, sz, P_C);
}

void report_timing_begin(vof_ctx* c, double snap[T_NCLASS]) {
    if (!c->timing) return;
    flush_timers(c);
    for (int t = 0; t < T_NCLASS; ++t) snap[t] = c->t_ms[t];
}

void report_timing_end(vof_ctx* c, const double snap[T_NCLASS], vof_report* r) {
    if (!c->timing || !r) return;
    flush_timers(c);
    double d[T_NCLASS];
    for (int t = 0; t < T_NCLASS; ++t) d[t] = c->t_ms[t] - snap[t];
    r->ms[0] = (float)d[T_ADVECT];
    r->ms[1] = (float)d[T_SSF];
    r->ms[2] = (float)d[T_PREDICT];
    r->ms[3] = (float)d[T_RHS];
    r->ms[4] = (float)(d[T_SMOOTH0] + d[T_SMOOTH] + d[T_RESIDUAL] + d[T_RESTRICT0] +
                       d[T_RESTRICT] + d[T_PROLONG0] + d[T_PROLONG] + d[T_COARSE] + d[T_KRYLOV]);
    r->ms[5] = (float)d[T_PROJECT];
    r->ms[6] = 0.f;
    double tot = 0;
    for (int t = 0; t < T_NCLASS; ++t) tot += d[t];
    r->ms[7] = (float)tot;
}

}  // namespace

size_t workspace_bytes(const vof_grid* g, const vof_solver* sv) {
    const Sizes s = sizes_of(g);
    const size_t faces = s.nu + s.nv + s.nw;
    size_t b = 0;
    b += 3 * faces * sizeof(double);                  // beta, surface force, fluxes
    b += s.n * sizeof(double);                        // kappa
    b += 3 * s.n;                                     // valid, cmask, has
    b += s.n * sizeof(int) + 64;                      // interface list
    b += s.n * (sizeof(int) + 1) + 512;               // its piece order and pieces
    b += 4 * s.n * sizeof(double);                    // planes
    b += 3 * s.n * sizeof(double);                    // cell intermediate velocity
    b += 3 * s.n * sizeof(double);                    // alpha scratch
    b += 6 * s.n * sizeof(double);                    // b, r, z, p, q, rhs
    b += mg_workspace_bytes(g, sv, nullptr);
    if (sv->precision == VOF_PREC_MIXED_FP32) b += 4 * s.n * sizeof(float);  // FP32 velocities, alpha
    if (sv->ssf_solves == 2) b += 2 * s.n * sizeof(double);                  // p~ and p
    b += (size_t)NSLOTS * MAX_PARTIALS * sizeof(double) + S_NSCALARS * sizeof(double) + 64;
    return b;
}

bool grid_ok(const vof_grid* g, std::string& why) {
    if (!g) { why = "grid is NULL"; return false; }
    if (g->nx < 2 || g->ny < 2 || g->nz < 4) { why = "need nx, ny >= 2 and nz >= 4"; return false; }
    if (g->nz % 2) { why = "nz must be even (red-black ordering on the periodic axis)"; return false; }
    if (!(g->h > 0.0) || !std::isfinite(g->h)) { why = "h must be positive"; return false; }
    if ((g->periodic_x && g->nx % 2) || (g->periodic_y && g->ny % 2)) {
        why = "periodic x/y need an even cell count";
        return false;
    }
    const double faces = (double)(g->nx + 1) * (double)(g->ny + 1) * (double)g->nz;
    if (faces >= 2147483647.0) { why = "grid too large for 32-bit indexing"; return false; }
    const long tiles = (long)((g->nx + TBX - 1) / TBX) * ((g->ny + TBY - 1) / TBY);
    if (tiles > MAX_PARTIALS) { why = "cross-section too large"; return false; }
    return true;
}

bool phys_ok(const vof_phys* p) {
    return p && p->rho_l > 0 && p->rho_g > 0 && p->mu_l >= 0 && p->mu_g >= 0 && p->sigma >= 0 &&
           (p->conv_scheme == VOF_CONV_CENTRAL || p->conv_scheme == VOF_CONV_UPWIND) &&
           (p->kappa_mode == VOF_KAPPA_HEIGHT_FUNCTION || p->kappa_mode == VOF_KAPPA_EXACT);
}

// ---------------------------------------------------------------------------
// helpers used by the other translation units
// ---------------------------------------------------------------------------
// Workspace comes from the stream-ordered allocator on the context's stream:
// freeing it does not synchronise the whole device, so contexts that come
// and go on other streams (the request server) do not stall each other.
void* dev_alloc(vof_ctx* c, size_t bytes) {
    if (c->arena) {  // carved from an ensemble's arena, in allocation order
        const size_t off = (c->arena_used + 255) & ~(size_t)255;
        if (off + bytes > c->arena_size) return nullptr;
        c->arena_used = off + bytes;
        return c->arena + off;
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, c->st) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    c->allocs.push_back(p);
    return p;
}

vof_status set_err(vof_ctx* c, vof_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

vof_status cuda_check(vof_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return VOF_OK;
    return set_err(c, VOF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

vof_status launch_check(vof_ctx* c, const char* what) {
    return cuda_check(c, cudaGetLastError(), what);
}

int timer_begin(vof_ctx* c, int cls) {
    if (!c->timing) return -1;
    if (c->ev_marks.size() >= 8192) flush_timers(c);
    const size_t need = 2 * (c->ev_marks.size() + 1);
    while (c->ev_pool.size() < need) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_pool.push_back(e);
    }
    const int a = (int)(2 * c->ev_marks.size()), b = a + 1;
    cudaEventRecord(c->ev_pool[a], c->st);
    c->ev_marks.push_back({cls, {a, b}});
    return (int)c->ev_marks.size() - 1;
}

void timer_end(vof_ctx* c, int, int mark) {
    if (mark < 0) return;
    cudaEventRecord(c->ev_pool[c->ev_marks[mark].second.second], c->st);
}

// copies of vof_step_host: the state's host arrays and device copies, in
// the order alpha, uc, vc, wc, u, v, w, p
struct StepIO {
    double* const* host;
    double* const* dev;
    size_t bytes[8];
};
enum { IO_ALPHA = 0, IO_UC, IO_VC, IO_WC, IO_U, IO_V, IO_W, IO_P };
// events of vof_step_host: inputs arrived (u, v, w, alpha; cell velocities;
// P), a point of the context stream where fields are final, copies out
// finished, start of the call
enum { EV_IN_FACES = 0, EV_IN_CELLS, EV_IN_P, EV_OUT_POINT, EV_OUT_DONE, EV_CALL };

// device-to-host copies of fields that the context stream has finished
// writing, on the copy-out stream once the stream's work so far is done;
// each copy records its field's event, which the next call's copy in of
// that field waits for
static void io_out(vof_ctx* c, const StepIO* io, std::initializer_list<int> fields) {
    if (!io) return;
    cudaEventRecord(c->io_ev[EV_OUT_POINT], c->st);
    cudaStreamWaitEvent(c->io_st[1], c->io_ev[EV_OUT_POINT], 0);
    for (int q : fields) {
        cudaMemcpyAsync(io->host[q], io->dev[q], io->bytes[q], cudaMemcpyDeviceToHost,
                        c->io_st[1]);
        cudaEventRecord(c->io_d2h[q], c->io_st[1]);
    }
}

// steps 11-12 on (u_hat_c in Uh, u_hat_f in u, v, w): right side, solve,
// correction of faces (in place) and cells (written to Uc)
static vof_status project_impl(vof_ctx* c, const double* const Uh[3], double* const Uc[3],
                               double* u, double* v, double* w, double* p, const double* sx,
                               const double* sy, const double* sz, double dt, vof_report* r,
                               const StepIO* io = nullptr) {
    vof_status st;
    if (io) cudaStreamWaitEvent(c->st, c->io_ev[EV_IN_P], 0);  // the guess P has arrived
    if (c->sv.ssf_solves == 2) {
        // the paper's steps 6 and 11: p~ from the surface force, p from the
        // velocity divergence, both with beta^{n+1}; P = p + p~. The guess
        // for p is P^n - p~^n; p~ starts from its previous solution.
        const int n = c->d.nx * c->d.ny * c->d.nz;
        launch_lincomb(c, n, 1.0, p, -1.0, c->ptilde, c->pflow);
        launch_rhs(c, u, v, w, sx, sy, sz, dt, c->rhs, 2);
        vof_report r1;
        std::memset(&r1, 0, sizeof(r1));
        st = solve_pressure(c, c->rhs, c->ptilde, &r1);
        if (st != VOF_OK && st != VOF_ERR_NOT_CONVERGED) return st;
        launch_rhs(c, u, v, w, sx, sy, sz, dt, c->rhs, 1);
        const vof_status st2 = solve_pressure(c, c->rhs, c->pflow, r);
        if (st2 != VOF_OK && st2 != VOF_ERR_NOT_CONVERGED) return st2;
        launch_lincomb(c, n, 1.0, c->pflow, 1.0, c->ptilde, p);
        r->iters += r1.iters;
        r->refinements += r1.refinements;
        r->res = std::max(r->res, r1.res);
        r->b_mean += r1.b_mean;
        st = st != VOF_OK ? st : st2;
    } else {
        launch_rhs(c, u, v, w, sx, sy, sz, dt, c->rhs, 3);
        st = solve_pressure(c, c->rhs, p, r);
        if (st != VOF_OK && st != VOF_ERR_NOT_CONVERGED) return st;
    }
    io_out(c, io, {IO_P});  // P is final; the correction only reads it
    launch_correct(c, p, sx, sy, sz, dt, Uh, Uc, u, v, w, P_A, P_B);
    io_out(c, io, {IO_U, IO_V, IO_W, IO_UC, IO_VC, IO_WC});
    readback(c);
    r->max_div = c->hbuf[S_MAXDIV];
    r->max_u = c->hbuf[S_MAXU];
    vof_status st2 = launch_check(c, "project");
    return st2 ? st2 : st;
}

// the whole time step. With io (vof_step_host) the fields are the device
// copies, whose inputs arrive on the copy-in stream: u, v, w and alpha
// before the call (the context stream already waits for them), the cell
// velocities before the predictor and P before the solve; each field is
// copied out as soon as the step has finished writing it.
static vof_status step_run(vof_ctx* c, double* alpha, double* uc, double* vc, double* wc,
                           double* u, double* v, double* w, double* p, double dt,
                           long long step_index, vof_report* report, const StepIO* io) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, uc);
    REQUIRE_PTR(c, vc);
    REQUIRE_PTR(c, wc);
    REQUIRE_PTR(c, u);
    REQUIRE_PTR(c, v);
    REQUIRE_PTR(c, w);
    REQUIRE_PTR(c, p);
    if ((st = walls_only(c, "step"))) return st;
    if (step_index < 0) return set_err(c, VOF_ERR_ARG, "step_index must be >= 0");
    if ((st = cfl_check(c, u, v, w, dt))) return st;
    double snap[T_NCLASS];
    report_timing_begin(c, snap);
    const size_t n = (size_t)c->d.nx * c->d.ny * c->d.nz;
    // steps 1-2: keep alpha^n (rho^n, mu^n) for the predictor
    cudaMemcpyAsync(c->an, alpha, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    // step 3: advect alpha with u_f^n, keeping the liquid face fluxes
    double* const flux[3] = {c->fx, c->fy, c->fz};
    advect_impl(c, alpha, u, v, w, dt, step_index, flux);
    io_out(c, io, {IO_ALPHA});  // alpha^{n+1} is final
    // step 4 (beta from alpha^{n+1}) and steps 5-7 (curvature, face force):
    // they read alpha^{n+1} only, so they run while the cell velocities may
    // still be arriving
    launch_beta(c, alpha);
    ssf_impl(c, alpha, c->kappa, c->sx, c->sy, c->sz);
    if (io) cudaStreamWaitEvent(c->st, c->io_ev[EV_IN_CELLS], 0);
    // steps 8-9: cell-centred intermediate velocity
    const double* const U[3] = {uc, vc, wc};
    launch_predict(c, c->an, alpha, U, u, v, w, c->fx, c->fy, c->fz, dt, c->uh);
    // step 10: face intermediate velocity
    launch_cell_to_face(c, c->uh[0], c->uh[1], c->uh[2], u, v, w);
    // steps 11-12
    vof_report r;
    std::memset(&r, 0, sizeof(r));
    const double* const Uh[3] = {c->uh[0], c->uh[1], c->uh[2]};
    double* const Uc[3] = {uc, vc, wc};
    st = project_impl(c, Uh, Uc, u, v, w, p, c->sx, c->sy, c->sz, dt, &r, io);
    if (report) {
        readback(c);
        fill_vof_report(c, &r);
        r.hf_fallbacks = (long long)llround(c->hbuf[S_FALLBACK]);
        *report = r;
        report_timing_end(c, snap, report);
    }
    return st;
}

// the whole time step behind step() and vof_step(); internal callers (the
// request server) use this name, never the exported one
vof_status step_entry(vof_ctx* c, double* alpha, double* uc, double* vc, double* wc, double* u,
                      double* v, double* w, double* p, double dt, long long step_index,
                      vof_report* report) {
    return step_run(c, alpha, uc, vc, wc, u, v, w, p, dt, step_index, report, nullptr);
}

// The ensemble's step around a batched pressure solve, for one case: step_pre
// launches step_run's kernels up to the pressure solve and the solve's setup
// (the guess P copied into the context's P workspace c->p); the batched solve
// (solve_mixed_batch) runs the solve of every case; step_post launches the
// rest. In sequence they launch the case's kernels of step_run, in its order,
// on the same values (the mixed single-solve path).
vof_status step_pre_cfl(vof_ctx* c, double* const f[8], double dt) {
    vof_status st = check_ctx(c);
    if (st) return st;
    for (int q = 0; q < 8; ++q)
        if (!f[q]) return set_err(c, VOF_ERR_ARG, "a field is NULL");
    if ((st = walls_only(c, "step"))) return st;
    if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(c, VOF_ERR_ARG, "dt must be positive");
    launch_cfl(c, f[4], f[5], f[6], dt, P_A);
    readback_async(c);
    return VOF_OK;
}

// after step_pre_cfl and a wait on the stream: cfl_check's test, then the
// rest of the step up to the solve
vof_status step_pre(vof_ctx* c, double* const f[8], double dt, long long step_index) {
    if (step_index < 0) return set_err(c, VOF_ERR_ARG, "step_index must be >= 0");
    const double cfl = c->hbuf[S_CFL] * dt / c->g.h;
    if (!std::isfinite(cfl)) return set_err(c, VOF_ERR_NONFINITE, "non-finite velocity");
    if (cfl > 1.0)
        return set_err(c, VOF_ERR_CFL, "Courant number " + std::to_string(cfl) + " exceeds 1");
    return step_pre_launch(c, f, dt, step_index);
}

vof_status step_pre_launch(vof_ctx* c, double* const f[8], double dt, long long step_index) {
    double* const alpha = f[0];
    const double *u = f[4], *v = f[5], *w = f[6];
    const size_t n = (size_t)c->d.nx * c->d.ny * c->d.nz;
    cudaMemcpyAsync(c->an, alpha, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    double* const flux[3] = {c->fx, c->fy, c->fz};
    advect_impl(c, alpha, u, v, w, dt, step_index, flux);
    launch_beta(c, alpha);
    ssf_impl(c, alpha, c->kappa, c->sx, c->sy, c->sz);
    const double* const U[3] = {f[1], f[2], f[3]};
    launch_predict(c, c->an, alpha, U, u, v, w, c->fx, c->fy, c->fz, dt, c->uh);
    launch_cell_to_face(c, c->uh[0], c->uh[1], c->uh[2], f[4], f[5], f[6]);
    launch_rhs(c, u, v, w, c->sx, c->sy, c->sz, dt, c->rhs, 3);
    launch_copy(c, c->p, f[7], (int)n);
    solve_setup_mixed(c, c->rhs, c->p);
    return launch_check(c, "step");
}

// solve: the status of the case's solve; its iteration counts are in
// *report. step_post launches the correction and the readback of its maxima
// without a wait; step_post_report, after a wait on the stream, fills the
// report and returns the step's status.
vof_status step_post(vof_ctx* c, double* const f[8], double dt, vof_status solve) {
    if (solve != VOF_OK && solve != VOF_ERR_NOT_CONVERGED) return solve;
    const int n = c->d.nx * c->d.ny * c->d.nz;
    launch_copy(c, f[7], c->p, n);
    const double* const Uh[3] = {c->uh[0], c->uh[1], c->uh[2]};
    double* const Uc[3] = {f[1], f[2], f[3]};
    launch_correct(c, f[7], c->sx, c->sy, c->sz, dt, Uh, Uc, f[4], f[5], f[6], P_A, P_B);
    readback_async(c);
    return solve;
}

vof_status step_post_report(vof_ctx* c, vof_status solve, vof_report* report) {
    if (solve != VOF_OK && solve != VOF_ERR_NOT_CONVERGED) return solve;
    vof_report r = report ? *report : vof_report{};
    r.max_div = c->hbuf[S_MAXDIV];
    r.max_u = c->hbuf[S_MAXU];
    const vof_status st2 = launch_check(c, "project");
    if (report) {
        fill_vof_report(c, &r);
        r.hf_fallbacks = (long long)llround(c->hbuf[S_FALLBACK]);
        *report = r;
    }
    return st2 ? st2 : solve;
}

// vof_step_host: the device copies of the state and the copy streams, made
// at the first call
static vof_status host_step_setup(vof_ctx* c) {
    if (!c->hs[0]) {
        const Sizes s = sizes_of(&c->g);
        const size_t n[8] = {s.n, s.n, s.n, s.n, s.nu, s.nv, s.nw, s.n};
        for (int q = 0; q < 8; ++q) {
            c->hs[q] = (double*)dev_alloc(c, n[q] * sizeof(double));
            if (!c->hs[q]) {
                for (int r = 0; r < q; ++r) {
                    cudaFreeAsync(c->hs[r], c->st);
                    c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), (void*)c->hs[r]));
                    c->hs[r] = nullptr;
                }
                return set_err(c, VOF_ERR_OOM, "vof_step_host: no device memory for the state");
            }
        }
    }
    // streams and events (each made once; a failed call is retried next time)
    cudaError_t e = cudaSuccess;
    for (auto& q : c->io_st)
        if (!q && e == cudaSuccess) e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
    for (auto& ev : c->io_ev)
        if (!ev && e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (auto& ev : c->io_d2h)
        if (!ev && e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    return cuda_check(c, e, "vof_step_host");
}


// ---------------------------------------------------------------------------
// the C ABI
// ---------------------------------------------------------------------------
extern "C" {

vof_status vof_workspace_bytes(const vof_grid* grid, const vof_solver* solver, size_t* bytes) {
    std::string why;
    if (!grid_ok(grid, why) || !bytes) return VOF_ERR_ARG;
    vof_solver def{VOF_PREC_FP64, 1e-10, 200, 2, 2, 0.0, 0, 0.0, VOF_MG_CONSTANT,
                   VOF_COARSEN_FACE_MEAN, VOF_CYCLE_W, 0, VOF_GRAPH_AUTO, 0, 1};
    *bytes = workspace_bytes(grid, solver ? solver : &def);
    return VOF_OK;
}

static vof_status create_impl(const vof_grid* grid, const vof_phys* phys,
                              const vof_solver* solver, size_t budget_bytes, void* stream,
                              char* arena, size_t arena_bytes, vof_ctx** out);

vof_status vof_create(const vof_grid* grid, const vof_phys* phys, const vof_solver* solver,
                      size_t budget_bytes, void* stream, vof_ctx** out) {
    return create_impl(grid, phys, solver, budget_bytes, stream, nullptr, 0, out);
}

}  // extern "C"

// a context whose workspace is carved from arena[0, arena_bytes) in a fixed
// order, so contexts made alike in equal arenas hold every array at the same
// offset (the ensemble's batched solve relies on it)
vof_status create_in_arena(const vof_grid* grid, const vof_phys* phys, const vof_solver* solver,
                           void* stream, void* arena, size_t arena_bytes, vof_ctx** out) {
    if (!arena || !arena_bytes) return VOF_ERR_ARG;
    return create_impl(grid, phys, solver, 0, stream, (char*)arena, arena_bytes, out);
}

static vof_status create_impl(const vof_grid* grid, const vof_phys* phys,
                              const vof_solver* solver, size_t budget_bytes, void* stream,
                              char* arena, size_t arena_bytes, vof_ctx** out) {
    if (!out) return VOF_ERR_ARG;
    *out = nullptr;
    std::string why;
    if (!grid_ok(grid, why) || !phys_ok(phys) || !solver) return VOF_ERR_ARG;
    if (!(solver->rtol > 0) || solver->max_iter < 1 || solver->nu_pre < 1 ||
        solver->nu_pre != solver->nu_post || !(solver->mg_omega >= 0.0) ||
        solver->mg_omega > 2.0 || solver->coarse_iters < 0 || !(solver->coarse_tol >= 0.0) ||
        (solver->mg_interp != VOF_MG_CONSTANT && solver->mg_interp != VOF_MG_TRILINEAR) ||
        (solver->mg_coarsen != VOF_COARSEN_FACE_MEAN &&
         solver->mg_coarsen != VOF_COARSEN_DENSITY_MEAN) ||
        (solver->mg_cycle != VOF_CYCLE_V && solver->mg_cycle != VOF_CYCLE_W) ||
        (solver->graph != VOF_GRAPH_AUTO && solver->graph != VOF_GRAPH_OFF &&
         solver->graph != VOF_GRAPH_CYCLE) ||
        (solver->mg_tail != VOF_TAIL_LAUNCHES && solver->mg_tail != VOF_TAIL_CLUSTER &&
         solver->mg_tail != VOF_TAIL_GRID) ||
        (solver->mg_tune != VOF_TUNE_AUTO && solver->mg_tune != VOF_TUNE_OFF) ||
        solver->mg_w_depth < 0 || solver->ssf_solves < 0 || solver->ssf_solves > 2 ||
        solver->nu_fine < 0 ||
        (solver->precision != VOF_PREC_FP64 && solver->precision != VOF_PREC_MIXED_FP32))
        return VOF_ERR_ARG;
    const size_t need = workspace_bytes(grid, solver);
    if (budget_bytes && need > budget_bytes) return VOF_ERR_ADMISSION;

    vof_ctx* c = new vof_ctx();
    c->arena = arena;
    c->arena_size = arena_bytes;
    c->g = *grid;
    c->ph = *phys;
    c->sv = *solver;
    c->d = Dims{grid->nx, grid->ny, grid->nz};
    c->st = (cudaStream_t)stream;
    c->bytes = need;
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->dev) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return VOF_ERR_CUDA;
    }
    c->Lc = launch_cells(grid->nx, grid->ny, grid->nz, c->sm_count);
    const Sizes s = sizes_of(grid);
    vof_status st = VOF_OK;
    auto A = [&](void** p, size_t b) {
        if (st == VOF_OK) st = alloc(c, p, b);
    };
    const size_t D = sizeof(double);
    A((void**)&c->bx, s.nu * D);
    A((void**)&c->by, s.nv * D);
    A((void**)&c->bz, s.nw * D);
    A((void**)&c->sx, s.nu * D);
    A((void**)&c->sy, s.nv * D);
    A((void**)&c->sz, s.nw * D);
    A((void**)&c->fx, s.nu * D);
    A((void**)&c->fy, s.nv * D);
    A((void**)&c->fz, s.nw * D);
    for (int q = 0; q < 3; ++q) A((void**)&c->uh[q], s.n * D);
    A((void**)&c->kappa, s.n * D);
    A((void**)&c->valid, s.n);
    A((void**)&c->cmask, s.n);
    A((void**)&c->has, s.n);
    A((void**)&c->if_list, s.n * sizeof(int));
    A((void**)&c->if_count, 64);
    A((void**)&c->if_perm, s.n * sizeof(int));
    A((void**)&c->if_piece, s.n);
    A((void**)&c->plane, 4 * s.n * D);
    A((void**)&c->a1, s.n * D);
    A((void**)&c->a2, s.n * D);
    A((void**)&c->an, s.n * D);
    A((void**)&c->b, s.n * D);
    A((void**)&c->r, s.n * D);
    A((void**)&c->z, s.n * D);
    A((void**)&c->p, s.n * D);
    A((void**)&c->q, s.n * D);
    A((void**)&c->rhs, s.n * D);
    A((void**)&c->part, (size_t)NSLOTS * MAX_PARTIALS * D);
    A((void**)&c->scal, S_NSCALARS * D);
    A((void**)&c->dflag, 64);
    if (c->sv.precision == VOF_PREC_MIXED_FP32)
        for (int q = 0; q < 4; ++q) A((void**)&c->u32[q], s.n * sizeof(float));
    if (c->sv.ssf_solves == 2) {
        A((void**)&c->ptilde, s.n * D);
        A((void**)&c->pflow, s.n * D);
    }
    if (st == VOF_OK) st = mg_allocate(c);
    if (st == VOF_OK && mg_tune_shapes(c, 1, 0, nullptr) != VOF_OK) {
        st = launch_check(c, "timing the multigrid launch shapes");
        if (st == VOF_OK) st = set_err(c, VOF_ERR_CUDA, "timing the multigrid launch shapes failed");
    }
    if (st == VOF_OK) {
        // the scalar mirror: a mapped page-locked slot, else pageable memory
        c->hbuf = mirror_acquire();
        if (c->hbuf && cudaHostGetDevicePointer((void**)&c->hmirror_dev, c->hbuf, 0) != cudaSuccess) {
            cudaGetLastError();
            mirror_release(c->hbuf);
            c->hbuf = nullptr;
            c->hmirror_dev = nullptr;
        }
        if (c->hbuf) std::memset(c->hbuf, 0, MIRROR_DOUBLES * sizeof(double));
        else c->hbuf = c->hbuf_store.data();
    }
    if (st == VOF_OK) {
        cudaMemsetAsync(c->scal, 0, S_NSCALARS * D, c->st);
        if (c->ptilde) cudaMemsetAsync(c->ptilde, 0, s.n * D, c->st);
        cudaMemsetAsync(c->part, 0, (size_t)NSLOTS * MAX_PARTIALS * D, c->st);
        st = cuda_check(c, cudaStreamSynchronize(c->st), "vof_create");
    }
    if (st != VOF_OK) {
        vof_destroy(c);
        return st;
    }
    *out = c;
    return VOF_OK;
}

extern "C" {

vof_status vof_destroy(vof_ctx* c) {
    if (!c) return VOF_ERR_ARG;
    for (cudaStream_t s : c->io_st)  // copies of vof_step_host still running
        if (s) cudaStreamSynchronize(s);
    cudaStreamSynchronize(c->st);
    for (void* p : c->allocs) cudaFreeAsync(p, c->st);
    cudaStreamSynchronize(c->st);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->vgraph) cudaGraphExecDestroy(c->vgraph);
    for (auto& sg : c->sgraph)
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
    for (cudaStream_t s : c->cap_st)
        if (s) cudaStreamDestroy(s);
    for (cudaStream_t s : c->io_st)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->io_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->io_d2h)
        if (e) cudaEventDestroy(e);
    if (c->hmirror_dev) mirror_release(c->hbuf);
    delete c;
    return VOF_OK;
}

const char* vof_last_error(const vof_ctx* c) {
    if (!c) return "NULL context";
    return c->err.c_str();
}

vof_status vof_advect(vof_ctx* c, double* alpha, const double* u, const double* v,
                      const double* w, double dt, long long step_index, double* fx, double* fy,
                      double* fz, vof_report* report) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, u);
    REQUIRE_PTR(c, v);
    REQUIRE_PTR(c, w);
    if (step_index < 0) return set_err(c, VOF_ERR_ARG, "step_index must be >= 0");
    if ((st = cfl_check(c, u, v, w, dt))) return st;
    double snap[T_NCLASS];
    report_timing_begin(c, snap);
    double* const flux[3] = {fx ? fx : c->fx, fy ? fy : c->fy, fz ? fz : c->fz};
    advect_impl(c, alpha, u, v, w, dt, step_index, flux);
    if ((st = launch_check(c, "vof_advect"))) return st;
    if (report) {
        readback(c);
        fill_vof_report(c, report);
        report_timing_end(c, snap, report);
        if ((st = launch_check(c, "vof_advect"))) return st;
    }
    return VOF_OK;
}

vof_status ssf_force(vof_ctx* c, const double* alpha, double* kappa, double* sx, double* sy,
                     double* sz) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, kappa);
    REQUIRE_PTR(c, sx);
    REQUIRE_PTR(c, sy);
    REQUIRE_PTR(c, sz);
    if ((st = walls_only(c, "ssf_force"))) return st;
    ssf_impl(c, alpha, kappa, sx, sy, sz);
    return launch_check(c, "ssf_force");
}

vof_status pressure_solve(vof_ctx* c, const double* alpha, const double* b, double* p,
                          vof_report* report) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, b);
    REQUIRE_PTR(c, p);
    if ((st = walls_only(c, "pressure_solve"))) return st;
    double snap[T_NCLASS];
    report_timing_begin(c, snap);
    launch_beta(c, alpha);
    vof_report r;
    std::memset(&r, 0, sizeof(r));
    st = solve_pressure(c, b, p, &r);
    if (report) {
        *report = r;
        report_timing_end(c, snap, report);
    }
    return st;
}

vof_status vof_apply_operator(vof_ctx* c, const double* alpha, const double* x, double* y) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, x);
    REQUIRE_PTR(c, y);
    if ((st = walls_only(c, "vof_apply_operator"))) return st;
    launch_beta(c, alpha);
    launch_apply_A(c, c->lv[0], x, y);
    return launch_check(c, "vof_apply_operator");
}

vof_status vof_predict(vof_ctx* c, const double* alpha_n, const double* alpha_np1, double* uc,
                       double* vc, double* wc, double* u, double* v, double* w, const double* fx,
                       const double* fy, const double* fz, double dt) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha_n);
    REQUIRE_PTR(c, alpha_np1);
    REQUIRE_PTR(c, uc);
    REQUIRE_PTR(c, vc);
    REQUIRE_PTR(c, wc);
    REQUIRE_PTR(c, u);
    REQUIRE_PTR(c, v);
    REQUIRE_PTR(c, w);
    REQUIRE_PTR(c, fx);
    REQUIRE_PTR(c, fy);
    REQUIRE_PTR(c, fz);
    if ((st = walls_only(c, "vof_predict"))) return st;
    if (!(dt > 0.0)) return set_err(c, VOF_ERR_ARG, "dt must be positive");
    const double* const U[3] = {uc, vc, wc};
    launch_predict(c, alpha_n, alpha_np1, U, u, v, w, fx, fy, fz, dt, c->uh);
    launch_cell_to_face(c, c->uh[0], c->uh[1], c->uh[2], u, v, w);
    const size_t n = (size_t)c->d.nx * c->d.ny * c->d.nz;
    cudaMemcpyAsync(uc, c->uh[0], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(vc, c->uh[1], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(wc, c->uh[2], n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    return launch_check(c, "vof_predict");
}

vof_status project(vof_ctx* c, const double* alpha, double* uc, double* vc, double* wc, double* u,
                   double* v, double* w, double* p, const double* sx, const double* sy,
                   const double* sz, double dt, vof_report* report) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, uc);
    REQUIRE_PTR(c, vc);
    REQUIRE_PTR(c, wc);
    REQUIRE_PTR(c, u);
    REQUIRE_PTR(c, v);
    REQUIRE_PTR(c, w);
    REQUIRE_PTR(c, p);
    REQUIRE_PTR(c, sx);
    REQUIRE_PTR(c, sy);
    REQUIRE_PTR(c, sz);
    if ((st = walls_only(c, "project"))) return st;
    if (!(dt > 0.0)) return set_err(c, VOF_ERR_ARG, "dt must be positive");
    double snap[T_NCLASS];
    report_timing_begin(c, snap);
    launch_beta(c, alpha);
    vof_report r;
    std::memset(&r, 0, sizeof(r));
    // the cell correction reads u_hat_c and writes u_c: keep a copy of u_hat_c
    const size_t n = (size_t)c->d.nx * c->d.ny * c->d.nz;
    cudaMemcpyAsync(c->uh[0], uc, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(c->uh[1], vc, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    cudaMemcpyAsync(c->uh[2], wc, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st);
    const double* const Uh[3] = {c->uh[0], c->uh[1], c->uh[2]};
    double* const Uc[3] = {uc, vc, wc};
    st = project_impl(c, Uh, Uc, u, v, w, p, sx, sy, sz, dt, &r);
    if (report) {
        *report = r;
        report_timing_end(c, snap, report);
    }
    return st;
}

vof_status step(vof_ctx* c, double* alpha, double* uc, double* vc, double* wc, double* u,
                double* v, double* w, double* p, double dt, long long step_index,
                vof_report* report) {
    return step_entry(c, alpha, uc, vc, wc, u, v, w, p, dt, step_index, report);
}

vof_status vof_step(vof_ctx* c, double* alpha, double* uc, double* vc, double* wc, double* u,
                    double* v, double* w, double* p, double dt, long long step_index,
                    vof_report* report) {
    return step_entry(c, alpha, uc, vc, wc, u, v, w, p, dt, step_index, report);
}

vof_status vof_step_host(vof_ctx* c, double* alpha, double* uc, double* vc, double* wc,
                         double* u, double* v, double* w, double* p, double dt,
                         long long step_index, vof_report* report) {
    vof_status st = check_ctx(c);
    if (st) return st;
    REQUIRE_PTR(c, alpha);
    REQUIRE_PTR(c, uc);
    REQUIRE_PTR(c, vc);
    REQUIRE_PTR(c, wc);
    REQUIRE_PTR(c, u);
    REQUIRE_PTR(c, v);
    REQUIRE_PTR(c, w);
    REQUIRE_PTR(c, p);
    if ((st = walls_only(c, "vof_step_host"))) return st;
    if ((st = host_step_setup(c))) return st;
    const Sizes s = sizes_of(&c->g);
    double* const host[8] = {alpha, uc, vc, wc, u, v, w, p};
    StepIO io{host, c->hs, {s.n * 8, s.n * 8, s.n * 8, s.n * 8, s.nu * 8, s.nv * 8, s.nw * 8,
                            s.n * 8}};
    // copies in after everything already on the context stream and, field
    // by field, after the previous call's copy out of the same field (those
    // run on in the background: the context stream does not wait for them).
    // alpha, u, v and w first: the CFL check and the advection need them;
    // alpha's copy out finished early in the previous call, u, v, w are the
    // previous call's first copies out after its projection. The cell
    // velocities and P come later.
    cudaStream_t in = c->io_st[0];
    cudaEventRecord(c->io_ev[EV_CALL], c->st);
    cudaStreamWaitEvent(in, c->io_ev[EV_CALL], 0);
    auto copy_in = [&](int q) {
        cudaStreamWaitEvent(in, c->io_d2h[q], 0);
        cudaMemcpyAsync(c->hs[q], host[q], io.bytes[q], cudaMemcpyHostToDevice, in);
    };
    for (int q : {IO_ALPHA, IO_U, IO_V, IO_W}) copy_in(q);
    cudaEventRecord(c->io_ev[EV_IN_FACES], in);
    for (int q : {IO_UC, IO_VC, IO_WC}) copy_in(q);
    cudaEventRecord(c->io_ev[EV_IN_CELLS], in);
    copy_in(IO_P);
    cudaEventRecord(c->io_ev[EV_IN_P], in);
    cudaStreamWaitEvent(c->st, c->io_ev[EV_IN_FACES], 0);
    if ((st = launch_check(c, "vof_step_host"))) return st;
    st = step_run(c, c->hs[IO_ALPHA], c->hs[IO_UC], c->hs[IO_VC], c->hs[IO_WC], c->hs[IO_U],
                  c->hs[IO_V], c->hs[IO_W], c->hs[IO_P], dt, step_index, report, &io);
    // with a report the call returns when every copy has finished
    if (report) {
        for (cudaStream_t q : c->io_st) cudaStreamSynchronize(q);
    }
    const vof_status st2 = launch_check(c, "vof_step_host");
    return st ? st : st2;
}

vof_status vof_diag_wait_timeout(vof_ctx* c) {
    vof_status st = check_ctx(c);
    if (st) return st;
    cudaMemsetAsync(c->scal + S_ERR, 0, sizeof(double), c->st);
    wait_probe(c, 1000);
    readback(c);
    const bool out = c->hbuf[S_ERR] != 0.0;
    cudaMemsetAsync(c->scal + S_ERR, 0, sizeof(double), c->st);  // the context stays usable
    if ((st = launch_check(c, "vof_diag_wait_timeout"))) return st;
    if (out) return set_err(c, VOF_ERR_TIMEOUT, "a bounded device wait ran out (diagnostic probe)");
    return VOF_OK;
}

vof_status vof_host_join(vof_ctx* c) {
    vof_status st = check_ctx(c);
    if (st) return st;
    for (cudaStream_t q : c->io_st) {
        if (!q) continue;
        cudaEventRecord(c->io_ev[EV_OUT_DONE], q);
        cudaStreamWaitEvent(c->st, c->io_ev[EV_OUT_DONE], 0);
    }
    return launch_check(c, "vof_host_join");
}

vof_status vof_launch_count(const vof_ctx* c, long long* n) {
    if (!c || !n) return VOF_ERR_ARG;
    *n = c->nlaunch;
    return VOF_OK;
}

vof_status vof_mg_shape(const vof_ctx* c, int level, int shape[4]) {
    return mg_shape_of(c, level, shape);
}

vof_status vof_mg_set_shape(vof_ctx* c, int level, const int shape[3]) {
    if (!c || !shape) return VOF_ERR_ARG;
    return mg_set_shape(c, level, shape);
}

vof_status vof_set_timing(vof_ctx* c, int on) {
    if (!c) return VOF_ERR_ARG;
    if (!on) flush_timers(c);
    c->timing = on ? 1 : 0;
    return VOF_OK;
}

vof_status vof_kernel_times(vof_ctx* c, const char** names, double* ms, long long* launches,
                            int cap, int* n) {
    static const char* kNames[T_NCLASS] = {
        "advect",   "ssf",         "predict",         "rhs",        "smooth_l0",
        "smooth",   "residual_l0", "restrict_l0",     "restrict",   "prolong_l0",
        "prolong",  "coarse",      "krylov",          "project"};
    if (!c || !n) return VOF_ERR_ARG;
    flush_timers(c);
    int k = 0;
    for (int t = 0; t < T_NCLASS && k < cap; ++t, ++k) {
        if (names) names[k] = kNames[t];
        if (ms) ms[k] = c->t_ms[t];
        if (launches) launches[k] = c->t_n[t];
        c->t_ms[t] = 0;
        c->t_n[t] = 0;
    }
    *n = k;
    return VOF_OK;
}

}  // extern "C"
