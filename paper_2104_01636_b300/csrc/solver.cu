// Pressure solve of Eq. 7 (steps 6/11): flexible conjugate gradients
// preconditioned by one symmetric geometric-multigrid V-cycle, the V-cycle
// in FP64 or (mixed precision) in FP32 while the residual, the operator,
// the dot products and the updates of P stay FP64.
//
// The paper relaxes with multigrid-accelerated red-black SOR (Section 2.1);
// here the same red-black relaxation is the smoother inside a V-cycle that
// preconditions a Krylov method. The V-cycle is symmetric (red-black
// before the coarse correction, black-red after; restriction is the scaled
// transpose of prolongation), so it is an SPD preconditioner; the flexible
// (A-orthogonalising) update keeps the outer iteration robust to the
// iteratively solved coarsest level.
#include <algorithm>
#include <cmath>

#include "vof_internal.cuh"

namespace {

bool can_coarsen(const Dims& d) {
    const long n = (long)d.nx * d.ny * d.nz;
    return n > 512 && d.nx % 2 == 0 && d.ny % 2 == 0 && d.nz % 2 == 0 && d.nx >= 4 && d.ny >= 4 &&
           d.nz >= 4;
}

std::vector<Dims> level_dims(const vof_grid* g) {
    std::vector<Dims> v;
    Dims d{g->nx, g->ny, g->nz};
    v.push_back(d);
    while (can_coarsen(d)) {
        d = Dims{d.nx / 2, d.ny / 2, d.nz / 2};
        v.push_back(d);
    }
    return v;
}

size_t faces_bytes(const Dims& d, size_t elt) {
    return elt * ((size_t)(d.nx + 1) * d.ny * d.nz + (size_t)d.nx * (d.ny + 1) * d.nz +
                  (size_t)d.nx * d.ny * d.nz);
}

template <class T>
void vcycle(vof_ctx* c, int l);
template <class T>
void cycle(vof_ctx* c, int l, bool zero_start);

// does level l visit its coarser level twice (W-cycle within mg_w_depth,
// default 3; never when the coarser level is the exactly solved coarsest)?
bool twice(const vof_ctx* c, int l) {
    const int depth = c->sv.mg_w_depth > 0 ? c->sv.mg_w_depth : 3;
    return c->sv.mg_cycle == VOF_CYCLE_W && l + 1 < (int)c->lv.size() - 1 && l < depth;
}

// Finest level of the mixed V-cycle with the density-formed coefficients:
// nu_pre red-black sweeps from a zero guess, restriction, the coarse
// correction, nu_post black-red sweeps. Sweeps ping-pong between xf and
// x32b; the pre-smoothing starts on the buffer that makes it end in xf.
// With sweep_dot the last sweep also forms (z, r) -> S_RZ and (z, q32) ->
// S_ZQ, the dots the flexible CG takes after every preconditioning.
void vcycle0_rho(vof_ctx* c) {
    Level& L0 = c->lv[0];
    float* const A = L0.xf;
    float* const B = c->x32b;
    const int nu = c->sv.nu_fine > 0 ? c->sv.nu_fine : c->sv.nu_pre;
    const float* cur = nullptr;  // zero
    float* dst = (nu % 2 == 1) ? A : B;
    for (int s = 0; s < nu; ++s) {
        rho_sweep(c, cur, dst, 0);
        cur = dst;
        dst = (dst == A) ? B : A;
    }
    rho_restrict(c);
    cycle<float>(c, 1, true);
    if (twice(c, 0)) cycle<float>(c, 1, false);
    mg_prolong<float>(c, c->lv[1], L0);
    for (int s = 0; s < nu; ++s) {
        rho_sweep(c, cur, dst, 1, c->sweep_dot && s == nu - 1);
        cur = dst;
        dst = (dst == A) ? B : A;
    }
    if (cur != A)
        cudaMemcpyAsync(A, cur, sizeof(float) * (size_t)L0.ncells, cudaMemcpyDeviceToDevice, c->st);
}

// symmetric multigrid cycle on the level arrays of type T (x <- M f at level
// l; zero_start false continues from the level's current x). A V-cycle
// visits the coarser level once; a W-cycle twice (the second visit
// continues from the first one's result; an exact coarsest solve is not
// repeated), which keeps the cycle symmetric.
template <class T>
void cycle(vof_ctx* c, int l, bool zero_start) {
    const Level& L = c->lv[l];
    if (sizeof(T) == sizeof(float) && l == c->tail_level && l > 0) {
        mg_tail_run(c, zero_start);  // this level and every coarser one, one launch
        return;
    }
    if (l == (int)c->lv.size() - 1) {
        mg_coarse<T>(c, L);
        return;
    }
    if (sizeof(T) == sizeof(float) && l == 0 && c->use_rho) {
        vcycle0_rho(c);
        return;
    }
    const int nu = (l == 0 && c->sv.nu_fine > 0) ? c->sv.nu_fine : c->sv.nu_pre;
    for (int s = 0; s < nu; ++s) {
        mg_rbgs<T>(c, L, 0, (s == 0 && zero_start) ? 1 : 0);  // from zero: no zeroing pass
        mg_rbgs<T>(c, L, 1);
    }
    mg_restrict<T>(c, L, c->lv[l + 1]);
    cycle<T>(c, l + 1, true);
    if (twice(c, l)) cycle<T>(c, l + 1, false);
    for (int s = 0; s < nu; ++s) {
        // the first pass adds the coarse correction to what it reads
        mg_rbgs<T>(c, L, 1, s == 0 ? 2 : 0, &c->lv[l + 1]);
        mg_rbgs<T>(c, L, 0);
    }
}

// The operations cycle<float>(c, l, zero_start) launches for a level l >= 1
// and everything below it, appended to a coarse-tail program in the same
// order (level indices relative to the tail level t0); false when the
// program does not fit.
bool tail_emit(const vof_ctx* c, int l, int t0, bool zero_start, TailProg& p) {
    auto push = [&](int kind, int lev, int color, int mode) {
        if (p.nops >= TAIL_MAX_OPS) return false;
        p.op[p.nops++] = TailOp{(unsigned char)kind, (unsigned char)(lev - t0),
                                (unsigned char)color, (unsigned char)mode};
        return true;
    };
    if (l == (int)c->lv.size() - 1) return push(TAIL_DENSE, l, 0, 0);
    const int nu = c->sv.nu_pre;
    for (int s = 0; s < nu; ++s)
        if (!push(TAIL_SMOOTH, l, 0, (s == 0 && zero_start) ? 1 : 0) || !push(TAIL_SMOOTH, l, 1, 0))
            return false;
    if (!push(TAIL_RESTRICT, l, 0, 0) || !tail_emit(c, l + 1, t0, true, p)) return false;
    if (twice(c, l) && !tail_emit(c, l + 1, t0, false, p)) return false;
    for (int s = 0; s < nu; ++s)
        if (!push(TAIL_SMOOTH, l, 1, s == 0 ? 2 : 0) || !push(TAIL_SMOOTH, l, 0, 0)) return false;
    return true;
}

// VOF_TAIL_CLUSTER on the mixed path with the dense coarsest solve: the
// first level l >= 1 of at most TAIL_MAX_CELLS cells runs its part of the
// cycle as one cluster launch per visit.
vof_status tail_setup(vof_ctx* c) {
    const int nl = (int)c->lv.size();
    if (c->sv.precision != VOF_PREC_MIXED_FP32 || c->sv.mg_interp != VOF_MG_CONSTANT ||
        c->dense_n <= 0 ||
        (c->sv.mg_tail != VOF_TAIL_CLUSTER && c->sv.mg_tail != VOF_TAIL_GRID))
        return VOF_OK;
    const bool grid = c->sv.mg_tail == VOF_TAIL_GRID;
    for (int t0 = 1; t0 + 1 < nl; ++t0) {
        if (c->lv[t0].ncells > (grid ? TAIL_GRID_MAX_CELLS : TAIL_MAX_CELLS) ||
            nl - t0 > TAIL_MAX_LEVELS)
            continue;
        // the FP16 coefficient copies of a large level are not the tail's
        if (c->lv[t0].bxh) continue;
        TailProg p[2];
        for (int z = 0; z < 2; ++z) {
            p[z] = TailProg{};
            p[z].omega = (float)(c->sv.mg_omega > 0.0 ? c->sv.mg_omega : 1.0);
            for (int l = t0; l < nl; ++l) {
                const Level& L = c->lv[l];
                p[z].L[l - t0] = TailLevel{L.d, (float)(L.h * L.h), (float)(1.0 / (L.h * L.h)),
                                           L.bxf, L.byf, L.bzf, L.xf, L.ff};
            }
        }
        if (tail_emit(c, t0, t0, true, p[0]) && tail_emit(c, t0, t0, false, p[1]))
            return mg_tail_setup(c, t0, &p[0], &p[1], grid);
    }
    return VOF_OK;
}

template <class T>
void vcycle(vof_ctx* c, int l) {
    cycle<T>(c, l, true);
}

// One V-cycle on the finest level's (x, f) in the context's precision. The
// first call captures the cycle's launches into a CUDA graph; later calls
// replay it, which removes the launch gaps between the small coarse-level
// kernels. The cycle reads only fixed workspace pointers (coefficients and
// the dense coarse inverse are refreshed in place each solve), so the graph
// stays valid for the context's lifetime. Per-kernel timing, or a stream
// that cannot be captured (the legacy default stream), keeps direct launches.
template <class T>
void run_vcycle(vof_ctx* c) {
    if (c->timing || c->vgraph_state < 0 || c->sv.graph == VOF_GRAPH_OFF || c->in_solve_capture) {
        vcycle<T>(c, 0);
        return;
    }
    if (c->vgraph_state == 0) {
        c->vgraph_state = -1;
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(c->st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
            cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            vcycle<T>(c, 0);
            return;
        }
        const long long n0 = c->nlaunch;
        vcycle<T>(c, 0);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->st, &g);
        c->vgraph_kernels = c->nlaunch - n0;
        c->nlaunch = n0;
        if (e != cudaSuccess || !g || cudaGraphInstantiate(&c->vgraph, g, 0) != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            c->vgraph = nullptr;
            vcycle<T>(c, 0);
            return;
        }
        cudaGraphDestroy(g);
        c->vgraph_state = 1;
    }
    cudaGraphLaunch(c->vgraph, c->st);
    c->nlaunch += c->vgraph_kernels;
}

// (z, r) -> S_RZ and (z, q) -> S_ZQ after z = M r on the mixed path; the
// fused last sweep has formed them already (with q32 as q: the first
// iteration of a refinement, which passes q = r, does not use (z, q))
void krylov_dots(vof_ctx* c, int n, const float* z, const float* r, const float* q) {
    if (c->use_rho && c->sweep_dot) return;
    k32_dot2(c, n, z, r, q);
}

// z = M r (one V-cycle), in the precision the context was created with
void precondition(vof_ctx* c) {
    Level& L0 = c->lv[0];
    if (c->sv.precision == VOF_PREC_FP64) {
        L0.x = c->z;
        L0.f = c->r;
        run_vcycle<double>(c);
    } else {
        mg_to_f32(c, c->r, L0.ff, L0.ncells);
        run_vcycle<float>(c);
        mg_to_f64(c, L0.xf, c->z, L0.ncells);
    }
}

}  // namespace

// does coarse level l of the mixed cycle keep FP16 copies of its coefficients?
static bool half_coef_level(const Dims& d, int l, const vof_solver* sv) {
    return l >= 1 && sv && sv->precision == VOF_PREC_MIXED_FP32 &&
           sv->mg_interp == VOF_MG_CONSTANT && d.nx % 2 == 0 &&
           (long)d.nx * d.ny * d.nz >= HALF_COEF_MIN_CELLS;
}

size_t mg_workspace_bytes(const vof_grid* g, const vof_solver* sv, int* nlevels) {
    std::vector<Dims> dims = level_dims(g);
    if (nlevels) *nlevels = (int)dims.size();
    const bool mixed = sv && sv->precision == VOF_PREC_MIXED_FP32;
    const bool rho = rho_path_eligible(g, sv, (int)dims.size());
    const size_t elt = mixed ? sizeof(float) : sizeof(double);
    size_t b = 0;
    for (size_t l = mixed ? 0 : 1; l < dims.size(); ++l) {
        const size_t n = (size_t)dims[l].nx * dims[l].ny * dims[l].nz;
        // the density-formed finest level keeps x, f, a second x and rho
        b += (l == 0 && rho) ? 4 * n * elt + 2 * n + 256 : faces_bytes(dims[l], elt) + 2 * n * elt;
        if (half_coef_level(dims[l], (int)l, sv)) b += faces_bytes(dims[l], sizeof(__half)) + 32;
    }
    if (mixed) b += 3 * (size_t)dims[0].nx * dims[0].ny * dims[0].nz * sizeof(float);  // e, p, q
    if (sv && sv->mg_interp == VOF_MG_TRILINEAR)  // residual scratch per non-coarsest level
        for (size_t l = 0; l + 1 < dims.size(); ++l)
            b += (size_t)dims[l].nx * dims[l].ny * dims[l].nz * elt;
    if (sv && sv->mg_coarsen == VOF_COARSEN_DENSITY_MEAN) {
        for (size_t l = 1; l < dims.size(); ++l)
            b += (size_t)dims[l].nx * dims[l].ny * dims[l].nz * elt;
        const size_t n0 = (size_t)dims[0].nx * dims[0].ny * dims[0].nz;
        if (!mixed) b += n0 * sizeof(double);  // FP64 finest-level density
        else if (!rho) b += n0 * sizeof(float);
    }
    const Dims& dc = dims.back();
    const size_t nc = (size_t)dc.nx * dc.ny * dc.nz;
    b += 4 * nc * sizeof(double);
    if (mixed) b += 2 * sizeof(TailProg);  // coarse-tail programs
    if (nc <= (size_t)DENSE_MAX) b += (nc * nc * 2 + 32 * 32 + 64 * nc) * elt;
    return b;
}

vof_status mg_allocate(vof_ctx* c) {
    std::vector<Dims> dims = level_dims(&c->g);
    c->lv.resize(dims.size());
    const bool mixed = c->sv.precision == VOF_PREC_MIXED_FP32;
    c->use_rho = rho_path_eligible(&c->g, &c->sv, (int)dims.size());
    double h = c->g.h;
    for (size_t l = 0; l < dims.size(); ++l) {
        Level& L = c->lv[l];
        L.idx = (int)l;
        L.d = dims[l];
        L.h = h;
        h *= 2.0;
        L.ncells = L.d.nx * L.d.ny * L.d.nz;
        L.L = launch_cells(L.d.nx, L.d.ny, L.d.nz, c->sm_count);
        if (l == 0) {
            L.bx = c->bx;
            L.by = c->by;
            L.bz = c->bz;
            if (!mixed) continue;
        }
        const size_t nu = (size_t)(L.d.nx + 1) * L.d.ny * L.d.nz;
        const size_t nv = (size_t)L.d.nx * (L.d.ny + 1) * L.d.nz;
        const size_t n = L.ncells;
        const size_t elt = mixed ? sizeof(float) : sizeof(double);
        if (l == 0 && c->use_rho) {
            // x, f, second x, FP32 density, then the FP16 density (n halves)
            float* q = (float*)dev_alloc(c, sizeof(float) * 4 * n + 2 * n + 256);
            if (!q) return set_err(c, VOF_ERR_OOM, "allocation of the finest level failed");
            L.xf = q;
            L.ff = q + n;
            c->x32b = q + 2 * n;
            c->rho32 = q + 3 * n;
            c->rho16 = (void*)(((uintptr_t)(q + 4 * n) + 255) & ~(uintptr_t)255);
            continue;
        }
        void* p = dev_alloc(c, elt * (nu + nv + 3 * n));
        if (!p) return set_err(c, VOF_ERR_OOM, "allocation of a multigrid level failed");
        if (mixed) {
            float* q = (float*)p;
            L.bxf = q;
            L.byf = q + nu;
            L.bzf = q + nu + nv;
            L.xf = q + nu + nv + n;
            L.ff = q + nu + nv + 2 * n;
            const double rmin = std::min(c->ph.rho_l, c->ph.rho_g);
            const double rmax = std::max(c->ph.rho_l, c->ph.rho_g);
            if (half_coef_level(L.d, (int)l, &c->sv) && rmin > 0.0 && rmax <= 8192.0 * rmin) {
                // every nonzero coefficient is a mean of 2/(rho_a + rho_b), so it
                // lies in [1/rmax, 1/rmin]; stored over s, the power of two at or
                // above 1/rmin, it lies in [2^-14, 1]: FP16's normal range
                L.hscale = (float)std::exp2(std::ceil(std::log2(1.0 / rmin)));
                // offsets rounded to 8 halves: the paired loads stay aligned
                const size_t ou = (nu + 7) & ~(size_t)7, ov = (nv + 7) & ~(size_t)7;
                __half* hq = (__half*)dev_alloc(c, sizeof(__half) * (ou + ov + n));
                if (!hq) return set_err(c, VOF_ERR_OOM, "allocation of a multigrid level failed");
                L.bxh = hq;
                L.byh = hq + ou;
                L.bzh = hq + ou + ov;
            }
        } else {
            double* q = (double*)p;
            L.bx = q;
            L.by = q + nu;
            L.bz = q + nu + nv;
            L.x = q + nu + nv + n;
            L.f = q + nu + nv + 2 * n;
        }
    }
    if (mixed) {
        float** inner[3] = {&c->e32, &c->p32, &c->q32};
        for (float** v : inner) {
            void* q = dev_alloc(c, sizeof(float) * (size_t)c->lv[0].ncells);
            if (!q) return set_err(c, VOF_ERR_OOM, "allocation of inner Krylov vectors failed");
            *v = (float*)q;
            // finite from the start: the fused dots read q32 before its first use
            cudaMemsetAsync(q, 0, sizeof(float) * (size_t)c->lv[0].ncells, c->st);
        }
    }
    if (c->sv.mg_interp == VOF_MG_TRILINEAR) {
        const size_t elt = mixed ? sizeof(float) : sizeof(double);
        for (size_t l = 0; l + 1 < c->lv.size(); ++l) {
            void* q = dev_alloc(c, elt * (size_t)c->lv[l].ncells);
            if (!q) return set_err(c, VOF_ERR_OOM, "allocation of a multigrid residual failed");
            c->lv[l].rs = q;
        }
    }
    if (c->sv.mg_coarsen == VOF_COARSEN_DENSITY_MEAN) {
        const size_t elt = mixed ? sizeof(float) : sizeof(double);
        for (size_t l = 1; l < c->lv.size(); ++l) {
            void* q = dev_alloc(c, elt * (size_t)c->lv[l].ncells);
            if (!q) return set_err(c, VOF_ERR_OOM, "allocation of a coarse density failed");
            c->lv[l].rho = q;
        }
        const size_t n0 = (size_t)c->lv[0].ncells;
        if (!mixed) {
            c->rho64 = (double*)dev_alloc(c, sizeof(double) * n0);
            if (!c->rho64) return set_err(c, VOF_ERR_OOM, "allocation of the density failed");
        } else if (!c->use_rho) {
            c->rho32 = (float*)dev_alloc(c, sizeof(float) * n0);
            if (!c->rho32) return set_err(c, VOF_ERR_OOM, "allocation of the density failed");
        }
    }
    const Level& Lc = c->lv.back();
    void* p = dev_alloc(c, 4 * sizeof(double) * (size_t)Lc.ncells);
    if (!p) return set_err(c, VOF_ERR_OOM, "allocation of the coarse scratch failed");
    c->coarse_scratch = (double*)p;
    if (Lc.ncells <= DENSE_MAX) {
        const size_t n2 = (size_t)Lc.ncells * Lc.ncells;
        const size_t elt = mixed ? sizeof(float) : sizeof(double);
        void* a = dev_alloc(c, n2 * elt);
        void* b = a ? dev_alloc(c, n2 * elt) : nullptr;
        void* w = b ? dev_alloc(c, (32 * 32 + 64 * (size_t)Lc.ncells) * elt) : nullptr;
        if (!a || !b || !w)
            return set_err(c, VOF_ERR_OOM, "allocation of the dense coarse inverse failed");
        c->dense_w = w;
        c->dense_a = (double*)a;
        c->dense_b = (double*)b;
        c->dense_n = Lc.ncells;
        // shift: the liquid face coefficient (the smallest physical one) per face
        c->dense_shift = 1.0 / c->ph.rho_l;
    }
    if (c->use_rho) {
        const vof_status st = rho_path_setup(c);
        if (st != VOF_OK) return st;
    }
    return tail_setup(c);
}

static void build_level_coefficients(vof_ctx* c);

void mg_build_coefficients(vof_ctx* c) {
    build_level_coefficients(c);
    mg_half_coefficients(c);
}

static void build_level_coefficients(vof_ctx* c) {
    const bool dens = c->sv.mg_coarsen == VOF_COARSEN_DENSITY_MEAN;
    if (dens && c->lv.size() > 1) {
        // coarse levels from the averaged density; the finest level keeps
        // its own coefficients (FP64 faces, their FP32 copies or rho32)
        const Level& L0 = c->lv[0];
        if (c->sv.precision == VOF_PREC_FP64) {
            mg_coarsen_density<double>(c, c->rho64, L0, c->lv[1]);
            for (size_t l = 2; l < c->lv.size(); ++l)
                mg_coarsen_density<double>(c, (const double*)c->lv[l - 1].rho, c->lv[l - 1], c->lv[l]);
            if (c->dense_n > 0) mg_dense_setup<double>(c, c->lv.back());
            return;
        }
        if (!c->use_rho) {
            const int nu = (L0.d.nx + 1) * L0.d.ny * L0.d.nz, nv = L0.d.nx * (L0.d.ny + 1) * L0.d.nz;
            mg_to_f32(c, c->bx, L0.bxf, nu);
            mg_to_f32(c, c->by, L0.byf, nv);
            mg_to_f32(c, c->bz, L0.bzf, L0.ncells);
        }
        mg_coarsen_density<float>(c, c->rho32, L0, c->lv[1]);
        for (size_t l = 2; l < c->lv.size(); ++l)
            mg_coarsen_density<float>(c, (const float*)c->lv[l - 1].rho, c->lv[l - 1], c->lv[l]);
        if (c->dense_n > 0 && !c->defer_dense) mg_dense_setup<float>(c, c->lv.back());
        return;
    }
    if (c->sv.precision == VOF_PREC_FP64) {
        for (size_t l = 1; l < c->lv.size(); ++l) mg_coarsen_beta<double>(c, c->lv[l - 1], c->lv[l]);
        if (c->dense_n > 0) mg_dense_setup<double>(c, c->lv.back());
        return;
    }
    const Level& L0 = c->lv[0];
    if (c->use_rho) {
        // the finest level forms its coefficients from rho32 (written with
        // the FP64 ones); level 1 averages the FP64 faces
        mg_coarsen_beta_from64(c, L0, c->lv[1]);
        for (size_t l = 2; l < c->lv.size(); ++l) mg_coarsen_beta<float>(c, c->lv[l - 1], c->lv[l]);
        if (c->dense_n > 0 && !c->defer_dense) mg_dense_setup<float>(c, c->lv.back());
        return;
    }
    const int nu = (L0.d.nx + 1) * L0.d.ny * L0.d.nz, nv = L0.d.nx * (L0.d.ny + 1) * L0.d.nz;
    mg_to_f32(c, c->bx, L0.bxf, nu);
    mg_to_f32(c, c->by, L0.byf, nv);
    mg_to_f32(c, c->bz, L0.bzf, L0.ncells);
    for (size_t l = 1; l < c->lv.size(); ++l) mg_coarsen_beta<float>(c, c->lv[l - 1], c->lv[l]);
    if (c->dense_n > 0 && !c->defer_dense) mg_dense_setup<float>(c, c->lv.back());
}

// Mixed precision: FP64 defect correction around an inner FP32 solve.
//   r = b - A64 P (FP64, stored also as FP32);  solve A32 e = r to a modest
//   relative tolerance with FP32 flexible CG preconditioned by the FP32
//   V-cycle;  P += e (FP64);  repeat until ||b - A64 P|| <= rtol ||b||.
// The residual, the update of P and every dot product stay FP64.
static vof_status solve_mixed(vof_ctx* c, double* P, double bnorm, double res0, vof_report* rep,
                              double b_mean) {
    Level& L0 = c->lv[0];
    const int n = L0.ncells;
    float* r32 = L0.ff;  // the inner residual is the V-cycle's fine right side
    float* z32 = L0.xf;  // and its output is the preconditioned residual
    double res = res0;
    int inner_total = 0, outer = 0;
    bool converged = res <= c->sv.rtol;
    while (!converged && inner_total < c->sv.max_iter && outer < 50) {
        // r32 holds the current FP64 residual rounded to FP32
        const double rr0 = res * bnorm * res * bnorm;
        const double tol_in = std::max(INNER_TOL_FLOOR, 0.2 * c->sv.rtol / res);
        // a stagnating FP32 inner solve must not use up the whole budget
        const int inner_cap = inner_total + std::max(20, c->sv.max_iter / 4);
        cudaMemsetAsync(c->e32, 0, sizeof(float) * (size_t)n, c->st);
        run_vcycle<float>(c);
        krylov_dots(c, n, z32, r32, r32);
        cudaMemcpyAsync(c->p32, z32, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, c->st);
        while (inner_total < c->sv.max_iter && inner_total < inner_cap) {
            ++inner_total;
            if (c->use_rho)
                rho_apply_A_dot(c, c->p32, c->q32, S_PQ);
            else
                k32_apply_A_dot(c, c->p32, c->q32, S_PQ);  // and alpha
            k32_cg_update(c, n, c->e32, r32, c->p32, c->q32, S_RR);
            readback(c);
            if (c->hbuf[S_ERR] != 0.0)
                return set_err(c, VOF_ERR_TIMEOUT, "a bounded device wait (TMA loads or a grid barrier) gave up");
            const double rr = c->hbuf[S_RR];
            if (!std::isfinite(rr)) return set_err(c, VOF_ERR_NONFINITE, "non-finite inner residual");
            if (rr <= tol_in * tol_in * rr0) break;
            run_vcycle<float>(c);
            krylov_dots(c, n, z32, r32, c->q32);  // and beta
            k32_p_update(c, n, c->p32, z32);
        }
        // FP64 update and true residual
        k32_add_to_f64(c, n, c->e32, P);
        launch_residual_to32(c, P, c->b, r32, S_RR);
        readback(c);
        res = std::sqrt(c->hbuf[S_RR]) / bnorm;
        if (c->hbuf[S_ERR] != 0.0)
            return set_err(c, VOF_ERR_TIMEOUT, "a bounded device wait (TMA loads or a grid barrier) gave up");
        if (!std::isfinite(res)) return set_err(c, VOF_ERR_NONFINITE, "non-finite residual");
        ++outer;
        converged = res <= c->sv.rtol;
    }
    launch_sub_mean(c, P, n, S_SUM);
    vof_status st = cuda_check(c, cudaGetLastError(), "pressure solve");
    if (rep) {
        rep->iters = inner_total;
        rep->refinements = outer;
        rep->res0 = res0;
        rep->res = res;
        rep->b_mean = b_mean;
    }
    if (st != VOF_OK) return st;
    if (!converged)
        return set_err(c, VOF_ERR_NOT_CONVERGED,
                       "pressure solve did not reach rtol within max_iter (res=" +
                           std::to_string(res) + ")");
    return VOF_OK;
}

// ---------------------------------------------------------------------------
// The mixed solve as one CUDA graph. The decisions the host loop of
// solve_mixed takes after each readback (inner convergence, the inner
// iteration cap, another refinement, errors) are taken on the device by
// single-thread control kernels that set the handles of two nested
// conditional WHILE nodes; the kernels of the solve and their order are those
// of solve_mixed, so the iterates are the same and the host waits once per
// solve instead of once per iteration. Every pass of either loop body adds
// one inner iteration, and both loops stop at max_iter (a guard counter
// stops them in any case), so the loops end.
// ---------------------------------------------------------------------------
namespace {

enum SolveStatus { ST_OK = 0, ST_TIMEOUT = 1, ST_NONFINITE = 2 };

struct SolveCtl {
    double rtol;
    int max_iter;
    int cap_add;  // inner iterations per refinement: max(20, max_iter / 4)
};

__global__ void k_ctl_setup(double* s, SolveCtl p, cudaGraphConditionalHandle h_out) {
    const double bb = s[S_BB];
    double bnorm = sqrt(bb);
    if (!(bnorm >= 1e-300)) bnorm = 1e-300;
    const bool zero = bb == 0.0;
    const double res0 = zero ? 0.0 : sqrt(s[S_RR]) / bnorm;
    s[S_BNORM] = bnorm;
    s[S_RES0] = res0;
    s[S_RES] = res0;
    s[S_INNER] = 0.0;
    s[S_OUTER] = 0.0;
    s[S_GUARD] = 0.0;
    s[S_ZERO] = zero ? 1.0 : 0.0;
    const int status = (!zero && !isfinite(res0)) ? ST_NONFINITE : ST_OK;
    s[S_STATUS] = status;
    const bool conv = zero || res0 <= p.rtol;
    s[S_CONV] = conv ? 1.0 : 0.0;
    cudaGraphSetConditional(h_out, (!conv && status == ST_OK) ? 1u : 0u);
}

__global__ void k_ctl_outer_begin(double* s, SolveCtl p) {
    const double res = s[S_RES], bnorm = s[S_BNORM];
    const double rr0 = res * bnorm * res * bnorm;
    const double tol_in = fmax(INNER_TOL_FLOOR, 0.2 * p.rtol / res);
    s[S_THR] = tol_in * tol_in * rr0;
    s[S_CAP] = s[S_INNER] + p.cap_add;
}

// after an inner CG update: count it, check the wait flag and the residual,
// and continue while the inner tolerance, max_iter and the cap allow
__global__ void k_ctl_inner(double* s, const double* __restrict__ part_rr, int nparts, SolveCtl p,
                            cudaGraphConditionalHandle h_in) {
    const double rr_sum = sum_partials(part_rr, nparts);  // (r, r), as finalize_sum forms it
    if (threadIdx.x != 0) return;
    s[S_RR] = rr_sum * 1.0;
    const double inner = s[S_INNER] + 1.0, guard = s[S_GUARD] + 1.0;
    s[S_INNER] = inner;
    s[S_GUARD] = guard;
    int status = (int)s[S_STATUS];
    if (s[S_ERR] != 0.0) status = ST_TIMEOUT;
    const double rr = s[S_RR];
    if (status == ST_OK && !isfinite(rr)) status = ST_NONFINITE;
    s[S_STATUS] = status;
    const bool cont = status == ST_OK && !(rr <= s[S_THR]) && inner < p.max_iter &&
                      inner < s[S_CAP] && guard < p.max_iter + 8;
    cudaGraphSetConditional(h_in, cont ? 1u : 0u);
}

// after the FP64 update and residual of a refinement
__global__ void k_ctl_outer_end(double* s, SolveCtl p, cudaGraphConditionalHandle h_out) {
    const double res = sqrt(s[S_RR]) / s[S_BNORM];
    s[S_RES] = res;
    int status = (int)s[S_STATUS];
    if (s[S_ERR] != 0.0) status = ST_TIMEOUT;
    if (status == ST_OK && !isfinite(res)) status = ST_NONFINITE;
    s[S_STATUS] = status;
    const double outer = s[S_OUTER] + 1.0;
    s[S_OUTER] = outer;
    const bool conv = res <= p.rtol;
    s[S_CONV] = conv ? 1.0 : 0.0;
    const bool cont = !conv && status == ST_OK && s[S_INNER] < p.max_iter && outer < 50.0 &&
                      s[S_GUARD] < p.max_iter + 8;
    cudaGraphSetConditional(h_out, cont ? 1u : 0u);
}

__global__ void k_zero_if(double* __restrict__ x, const double* __restrict__ s, int n) {
    if (s[S_ZERO] == 0.0) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        x[i] = 0.0;
}

// the graph being captured on stream s
cudaGraph_t capture_graph(cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return nullptr;
    return g;
}

// appends a conditional node (WHILE or IF) on handle h after the work
// captured so far on s; later captures on s follow the node; returns its body
// graph
cudaGraph_t capture_cond(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd) != cudaSuccess ||
        cs != cudaStreamCaptureStatusActive)
        return nullptr;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, deps, edges, nd, &np) != cudaSuccess) return nullptr;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies) != cudaSuccess)
        return nullptr;
    return np.conditional.phGraph_out[0];
}

cudaGraph_t capture_while(cudaStream_t s, cudaGraphConditionalHandle h) {
    return capture_cond(s, h, cudaGraphCondTypeWhile);
}

// the first CG step of a refinement or the later ones: z = M r, the
// direction, q = A p and the update of e and r, then the inner control
void inner_tail(vof_ctx* c, const SolveCtl& p, cudaGraphConditionalHandle h_in) {
    const int n = c->lv[0].ncells;
    if (c->use_rho)
        rho_apply_A_dot(c, c->p32, c->q32, S_PQ);
    else
        k32_apply_A_dot(c, c->p32, c->q32, S_PQ);  // and alpha
    const int nb = k32_cg_update(c, n, c->e32, c->lv[0].ff, c->p32, c->q32, S_RR, false);
    ++c->nlaunch;
    k_ctl_inner<<<1, 1024, 0, c->st>>>(c->scal, c->part + (size_t)S_RR * MAX_PARTIALS, nb, p, h_in);
}

// Captures the whole mixed solve for right side b_in and solution P into
// the graph slot sg. False (nothing left captured, the error cleared) when
// stream capture or conditional nodes are unavailable.
bool build_solve_graph(vof_ctx* c, vof_ctx::SolveGraph& sg, const double* b_in, double* P) {
    Level& L0 = c->lv[0];
    const int n = L0.ncells;
    float* r32 = L0.ff;
    float* z32 = L0.xf;
    cudaStream_t st0 = c->st;
    for (cudaStream_t& s : c->cap_st)
        if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st0, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
        cudaStreamBeginCapture(st0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const long long n0 = c->nlaunch;
    long long k_outer = 0, k_inner = 0;
    const SolveCtl p{c->sv.rtol, c->sv.max_iter, std::max(20, c->sv.max_iter / 4)};
    bool ok = true;
    c->in_solve_capture = true;
    cudaGraph_t g_top = capture_graph(st0);
    cudaGraphConditionalHandle h_out = 0, h_in = 0;
    ok = ok && g_top && cudaGraphConditionalHandleCreate(&h_out, g_top, 0,
                                                         cudaGraphCondAssignDefault) == cudaSuccess;
    // setup: b, its mean and norm, the initial FP64 residual
    cudaMemsetAsync(c->scal + S_ERR, 0, sizeof(double), st0);
    launch_copy(c, c->b, b_in, n);
    launch_sub_mean(c, c->b, n, S_MEAN);
    launch_dot(c, c->b, c->b, n, S_BB);
    launch_residual_to32(c, P, c->b, r32, S_RR);
    ++c->nlaunch;
    k_ctl_setup<<<1, 1, 0, st0>>>(c->scal, p, h_out);
    cudaGraph_t g_out = ok ? capture_while(st0, h_out) : nullptr;
    ok = ok && g_out;
    if (ok) {
        // one refinement: the inner FP32 solve of A e = r, then P += e and
        // the FP64 residual
        const long long m0 = c->nlaunch;
        c->st = c->cap_st[0];
        ok = cudaStreamBeginCaptureToGraph(c->st, g_out, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess &&
             cudaGraphConditionalHandleCreate(&h_in, g_out, 0, cudaGraphCondAssignDefault) ==
                 cudaSuccess;
        if (ok) {
            ++c->nlaunch;
            k_ctl_outer_begin<<<1, 1, 0, c->st>>>(c->scal, p);
            cudaMemsetAsync(c->e32, 0, sizeof(float) * (size_t)n, c->st);
            vcycle<float>(c, 0);
            krylov_dots(c, n, z32, r32, r32);
            cudaMemcpyAsync(c->p32, z32, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, c->st);
            inner_tail(c, p, h_in);
            cudaGraph_t g_in = capture_while(c->st, h_in);
            ok = g_in != nullptr;
            if (ok) {
                const long long i0 = c->nlaunch;
                c->st = c->cap_st[1];
                ok = cudaStreamBeginCaptureToGraph(c->st, g_in, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    vcycle<float>(c, 0);
                    krylov_dots(c, n, z32, r32, c->q32);  // and beta
                    k32_p_update(c, n, c->p32, z32);
                    inner_tail(c, p, h_in);
                    cudaGraph_t gb = nullptr;
                    ok = cudaStreamEndCapture(c->st, &gb) == cudaSuccess;
                }
                c->st = c->cap_st[0];
                k_inner = c->nlaunch - i0;
            }
            k32_add_to_f64(c, n, c->e32, P);
            launch_residual_to32(c, P, c->b, r32, S_RR);
            ++c->nlaunch;
            k_ctl_outer_end<<<1, 1, 0, c->st>>>(c->scal, p, h_out);
            cudaGraph_t gb = nullptr;
            ok = (cudaStreamEndCapture(c->st, &gb) == cudaSuccess) && ok;
        }
        c->st = st0;
        k_outer = c->nlaunch - m0 - k_inner;
    }
    // P = 0 for a zero right side, then mean-free
    ++c->nlaunch;
    k_zero_if<<<4 * c->sm_count, 256, 0, st0>>>(P, c->scal, n);
    launch_sub_mean(c, P, n, S_SUM);
    c->in_solve_capture = false;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st0, &g);
    const long long k_all = c->nlaunch - n0;
    c->nlaunch = n0;
    if (sg.exec) {
        cudaGraphExecDestroy(sg.exec);
        sg.exec = nullptr;
    }
    ok = ok && e == cudaSuccess && g && cudaGraphInstantiate(&sg.exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (!ok) {
        if (sg.exec) cudaGraphExecDestroy(sg.exec);
        sg.exec = nullptr;
        return false;
    }
    sg.b = b_in;
    sg.P = P;
    sg.k_outer = k_outer;
    sg.k_inner = k_inner;
    sg.k_fixed = k_all - k_outer - k_inner;
    return true;
}

// The mixed solve through its captured graph: one launch, one readback.
vof_status solve_mixed_graph(vof_ctx* c, const vof_ctx::SolveGraph& sg, vof_report* rep) {
    cudaGraphLaunch(sg.exec, c->st);
    readback(c);
    const long long inner = (long long)c->hbuf[S_INNER], outer = (long long)c->hbuf[S_OUTER];
    c->nlaunch += sg.k_fixed + outer * sg.k_outer + (inner - outer) * sg.k_inner;
    vof_status st = cuda_check(c, cudaGetLastError(), "pressure solve");
    if (rep) {
        rep->iters = (int)inner;
        rep->refinements = (int)outer;
        rep->res0 = c->hbuf[S_RES0];
        rep->res = c->hbuf[S_RES];
        rep->b_mean = c->hbuf[S_MEAN];
    }
    if (st != VOF_OK) return st;
    const int status = (int)c->hbuf[S_STATUS];
    if (status == ST_TIMEOUT)
        return set_err(c, VOF_ERR_TIMEOUT, "a bounded device wait (TMA loads or a grid barrier) gave up");
    if (status == ST_NONFINITE) return set_err(c, VOF_ERR_NONFINITE, "non-finite residual");
    if (c->hbuf[S_CONV] == 0.0)
        return set_err(c, VOF_ERR_NOT_CONVERGED,
                       "pressure solve did not reach rtol within max_iter (res=" +
                           std::to_string(c->hbuf[S_RES]) + ")");
    return VOF_OK;
}

// the cached graph for (b_in, P), captured on first use (the least recently
// used of the two slots is replaced); nullptr when capture is unavailable
const vof_ctx::SolveGraph* solve_graph_for(vof_ctx* c, const double* b_in, double* P) {
    ++c->sgraph_clock;
    for (auto& sg : c->sgraph)
        if (sg.exec && sg.b == b_in && sg.P == P) {
            sg.used = c->sgraph_clock;
            return &sg;
        }
    auto& slot = c->sgraph[0].used <= c->sgraph[1].used ? c->sgraph[0] : c->sgraph[1];
    if (!build_solve_graph(c, slot, b_in, P)) {
        c->sgraph_state = -1;
        return nullptr;
    }
    c->sgraph_state = 1;
    slot.used = c->sgraph_clock;
    return &slot;
}

}  // namespace

cudaGraph_t capture_if(cudaStream_t s, cudaGraphConditionalHandle h) {
    return capture_cond(s, h, cudaGraphCondTypeIf);
}

cudaGraph_t capture_graph_of(cudaStream_t s) { return capture_graph(s); }

void solve_tail_captured(vof_ctx* c) {
    const int n = c->lv[0].ncells;
    ++c->nlaunch;
    k_zero_if<<<4 * c->sm_count, 256, 0, c->st>>>(c->p, c->scal, n);
    launch_sub_mean(c, c->p, n, S_SUM);
}

// A right side that is exactly zero after its mean is removed has the
// mean-free solution P = 0.
static vof_status zero_solution(vof_ctx* c, double* P, vof_report* rep, double b_mean) {
    launch_zero(c, P, c->lv[0].ncells);
    if (rep) {
        rep->iters = 0;
        rep->refinements = 0;
        rep->res0 = 0.0;
        rep->res = 0.0;
        rep->b_mean = b_mean;
    }
    return cuda_check(c, cudaGetLastError(), "pressure solve");
}

// Solves A P = b_in - mean(b_in) with the fine-level beta already built.
vof_status solve_pressure(vof_ctx* c, const double* b_in, double* P, vof_report* rep) {
    const int n = c->lv[0].ncells;
    Level& L0 = c->lv[0];
    mg_build_coefficients(c);
    if (c->sv.precision == VOF_PREC_MIXED_FP32 && !c->timing && c->sv.graph == VOF_GRAPH_AUTO &&
        c->sgraph_state >= 0) {
        // the kernels are captured with the coarsest inverse and the
        // coefficients in place, which mg_build_coefficients refreshes in
        // place before every launch of the graph
        const vof_ctx::SolveGraph* sg = solve_graph_for(c, b_in, P);
        if (sg) return solve_mixed_graph(c, *sg, rep);
    }
    if (c->sv.precision == VOF_PREC_MIXED_FP32) {
        cudaMemsetAsync(c->scal + S_ERR, 0, sizeof(double), c->st);
        launch_copy(c, c->b, b_in, n);
        launch_sub_mean(c, c->b, n, S_MEAN);
        launch_dot(c, c->b, c->b, n, S_BB);
        launch_residual_to32(c, P, c->b, L0.ff, S_RR);
        readback(c);
        vof_status st = cuda_check(c, cudaGetLastError(), "pressure solve setup");
        if (st != VOF_OK) return st;
        if (c->hbuf[S_BB] == 0.0) return zero_solution(c, P, rep, c->hbuf[S_MEAN]);
        double bnorm = std::sqrt(c->hbuf[S_BB]);
        if (!(bnorm >= 1e-300)) bnorm = 1e-300;
        const double res0 = std::sqrt(c->hbuf[S_RR]) / bnorm;
        if (!std::isfinite(res0)) return set_err(c, VOF_ERR_NONFINITE, "non-finite initial residual");
        return solve_mixed(c, P, bnorm, res0, rep, c->hbuf[S_MEAN]);
    }

    launch_copy(c, c->b, b_in, n);
    launch_sub_mean(c, c->b, n, S_MEAN);
    launch_dot(c, c->b, c->b, n, S_BB);
    launch_residual(c, L0, P, c->b, c->r, S_RR);
    readback(c);
    vof_status st = cuda_check(c, cudaGetLastError(), "pressure solve setup");
    if (st != VOF_OK) return st;
    const double b_mean = c->hbuf[S_MEAN];
    if (c->hbuf[S_BB] == 0.0) return zero_solution(c, P, rep, b_mean);
    double bnorm = std::sqrt(c->hbuf[S_BB]);
    if (!(bnorm >= 1e-300)) bnorm = 1e-300;
    double res = std::sqrt(c->hbuf[S_RR]) / bnorm;
    const double res0 = res;
    if (!std::isfinite(res)) return set_err(c, VOF_ERR_NONFINITE, "non-finite initial residual");
    const double rtol = c->sv.rtol;
    int it = 0;
    int restarts = 0;
    bool converged = res <= rtol;
    while (!converged && it < c->sv.max_iter && restarts < 4) {
        // (re)start: z = M r, p = z
        precondition(c);
        launch_dot2(c, n, c->z, c->r, c->r, S_RZ, S_ZQ);
        launch_copy(c, c->p, c->z, n);
        while (it < c->sv.max_iter) {
            ++it;
            launch_apply_A_dot(c, L0, c->p, c->q, S_PQ);
            launch_scalar_alpha(c);
            launch_cg_update(c, n, P, c->r, c->p, c->q, S_RR);
            readback(c);
            res = std::sqrt(c->hbuf[S_RR]) / bnorm;
            if (!std::isfinite(res)) return set_err(c, VOF_ERR_NONFINITE, "non-finite residual");
            if (res <= rtol) break;
            precondition(c);
            launch_dot2(c, n, c->z, c->r, c->q, S_RZ, S_ZQ);
            launch_scalar_beta(c);
            launch_p_update(c, n, c->p, c->z);
        }
        // confirm with the true residual (the recursive one drifts)
        launch_residual(c, L0, P, c->b, c->r, S_RR);
        readback(c);
        res = std::sqrt(c->hbuf[S_RR]) / bnorm;
        converged = res <= rtol;
        ++restarts;
    }
    launch_sub_mean(c, P, n, S_SUM);
    st = cuda_check(c, cudaGetLastError(), "pressure solve");
    if (rep) {
        rep->iters = it;
        rep->refinements = 0;
        rep->res0 = res0;
        rep->res = res;
        rep->b_mean = b_mean;
    }
    if (st != VOF_OK) return st;
    if (!converged)
        return set_err(c, VOF_ERR_NOT_CONVERGED,
                       "pressure solve did not reach rtol within max_iter (res=" +
                           std::to_string(res) + ")");
    return VOF_OK;
}

// ---------------------------------------------------------------------------
// The ensemble's pressure solves as one batched solve. The cases' contexts
// were carved from one arena, so every launch of case 0's context m runs for
// all cases at once (bat_n cases, bat_stride bytes apart). The loop below is
// solve_mixed's, taken for every case on the host after one readback of all
// cases' scalars; a case whose loop has ended is switched off in the device
// flags, and its blocks return at once in every batched kernel. Each case's
// kernels, blocks, sums and decisions are those of its solo solve_mixed, so
// its iterates are the same bits.
// ---------------------------------------------------------------------------
void solve_setup_mixed(vof_ctx* c, const double* b_in, double* P) {
    const int n = c->lv[0].ncells;
    mg_build_coefficients(c);
    cudaMemsetAsync(c->scal + S_ERR, 0, sizeof(double), c->st);
    launch_copy(c, c->b, b_in, n);
    launch_sub_mean(c, c->b, n, S_MEAN);
    launch_dot(c, c->b, c->b, n, S_BB);
    launch_residual_to32(c, P, c->b, c->lv[0].ff, S_RR);
}

struct BatchSolveState {
    int nc = 0;
    int* act_h = nullptr;     // page-locked: the flags to push
    int* act_d = nullptr;     // device flags the batched kernels read
    double* mir_h = nullptr;  // mapped: nc x MIRROR_DOUBLES scalars
    double* mir_d = nullptr;
    long long* trips_h = nullptr;  // mapped: passes of the captured loop bodies (outer, inner)
    long long* trips_d = nullptr;
};

bool batch_solve_eligible(const vof_ctx* c) {
    if (c->sv.precision != VOF_PREC_MIXED_FP32 || !c->use_rho || !c->sweep_dot ||
        c->sv.mg_interp != VOF_MG_CONSTANT || c->sv.mg_coarsen != VOF_COARSEN_FACE_MEAN ||
        c->dense_n <= 0 || c->tail_level != 0 || c->sv.ssf_solves == 2 || c->timing)
        return false;
    const int nu = c->sv.nu_fine > 0 ? c->sv.nu_fine : c->sv.nu_pre;
    if (nu % 2 != 0 || c->lv[0].ncells % 4 != 0) return false;  // the finest sweeps end in xf
    for (size_t l = 1; l + 1 < c->lv.size(); ++l)
        if (c->lv[l].d.nx % 2 != 0) return false;  // the pair kernels on every smoothed level
    return true;
}

BatchSolveState* batch_solve_create(vof_ctx* m, int nc, long long stride) {
    BatchSolveState* b = new BatchSolveState();
    b->nc = nc;
    bool ok = cudaHostAlloc((void**)&b->act_h, sizeof(int) * nc, cudaHostAllocPortable) ==
                  cudaSuccess &&
              cudaMalloc((void**)&b->act_d, sizeof(int) * nc) == cudaSuccess &&
              cudaHostAlloc((void**)&b->mir_h, sizeof(double) * MIRROR_DOUBLES * nc,
                            cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&b->mir_d, b->mir_h, 0) == cudaSuccess &&
              cudaHostAlloc((void**)&b->trips_h, 2 * sizeof(long long),
                            cudaHostAllocMapped | cudaHostAllocPortable) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&b->trips_d, b->trips_h, 0) == cudaSuccess;
    ok = ok && rho_path_batch_maps(m, nc, stride) == VOF_OK;
    if (!ok) {
        cudaGetLastError();
        batch_solve_destroy(b);
        return nullptr;
    }
    return b;
}

vof_status batch_solve_tune(vof_ctx* m, BatchSolveState* b, long long stride) {
    return mg_tune_shapes(m, b->nc, stride, b->act_d);
}

void batch_solve_destroy(BatchSolveState* b) {
    if (!b) return;
    if (b->act_h) cudaFreeHost(b->act_h);
    if (b->act_d) cudaFree(b->act_d);
    if (b->mir_h) cudaFreeHost(b->mir_h);
    if (b->trips_h) cudaFreeHost(b->trips_h);
    delete b;
}

namespace {
struct CaseSolve {
    bool outer = false, inner = false, conv = false, err = false, zero = false;
    double bnorm = 1.0, res = 0.0, res0 = 0.0, rr0 = 0.0, tol_in = 0.0;
    int inner_total = 0, outer_n = 0, cap = 0;
};
}  // namespace

vof_status solve_mixed_batch(vof_ctx* m, int nc, long long stride, const int* run,
                             BatchSolveState* bs, vof_status* status, vof_report* reps,
                             vof_ctx* const* cases) {
    Level& L0 = m->lv[0];
    const int n = L0.ncells;
    float* r32 = L0.ff;
    float* z32 = L0.xf;
    const double rtol = m->sv.rtol;
    const int max_iter = m->sv.max_iter;
    std::vector<CaseSolve> cs(nc);
    m->bat_n = nc;
    m->bat_stride = stride;
    m->bat_act = bs->act_d;
    auto S = [&](int i, int slot) { return bs->mir_h[(size_t)i * MIRROR_DOUBLES + slot]; };
    auto push = [&](bool CaseSolve::*flag) {
        int any = 0;
        for (int i = 0; i < nc; ++i) any |= (bs->act_h[i] = (cs[i].*flag && !cs[i].err) ? 1 : 0);
        cudaMemcpyAsync(bs->act_d, bs->act_h, sizeof(int) * nc, cudaMemcpyHostToDevice, m->st);
        return any != 0;
    };
    auto fail = [&](int i, vof_status st, const char* msg) {
        cs[i].err = true;
        cs[i].outer = cs[i].inner = false;
        status[i] = set_err(cases[i], st, msg);
    };
    // the dense coarsest inverses of all cases (their coefficients were built
    // by each case's setup), one launch per Gauss-Jordan block step
    for (int i = 0; i < nc; ++i) bs->act_h[i] = run[i] ? 1 : 0;
    cudaMemcpyAsync(bs->act_d, bs->act_h, sizeof(int) * nc, cudaMemcpyHostToDevice, m->st);
    if (m->defer_dense) mg_dense_setup<float>(m, m->lv.back());
    readback_batch(m, bs->mir_d);
    for (int i = 0; i < nc; ++i) {
        status[i] = VOF_OK;
        if (!run[i]) {
            cs[i].err = true;
            continue;
        }
        reps[i].iters = 0;
        reps[i].refinements = 0;
        reps[i].b_mean = S(i, S_MEAN);
        const double bb = S(i, S_BB);
        if (bb == 0.0) {  // P = 0, as zero_solution
            cs[i].zero = true;
            reps[i].res0 = reps[i].res = 0.0;
            continue;
        }
        double bnorm = std::sqrt(bb);
        if (!(bnorm >= 1e-300)) bnorm = 1e-300;
        cs[i].bnorm = bnorm;
        cs[i].res0 = cs[i].res = std::sqrt(S(i, S_RR)) / bnorm;
        if (!std::isfinite(cs[i].res0)) {
            fail(i, VOF_ERR_NONFINITE, "non-finite initial residual");
            continue;
        }
        cs[i].conv = cs[i].res <= rtol;
        cs[i].outer = !cs[i].conv;
    }
    for (;;) {
        for (auto& q : cs)
            if (q.outer && !(q.inner_total < max_iter && q.outer_n < 50)) q.outer = false;
        for (auto& q : cs)
            if (q.outer) {
                q.rr0 = q.res * q.bnorm * q.res * q.bnorm;
                q.tol_in = std::max(INNER_TOL_FLOOR, 0.2 * rtol / q.res);
                q.cap = q.inner_total + std::max(20, max_iter / 4);
                q.inner = true;
            }
        if (!push(&CaseSolve::outer)) break;
        launch_zero32_bat(m, m->e32, n);
        run_vcycle<float>(m);
        krylov_dots(m, n, z32, r32, r32);
        launch_copy32_bat(m, m->p32, z32, n);
        for (;;) {
            for (auto& q : cs)
                if (q.inner && !(q.inner_total < max_iter && q.inner_total < q.cap)) q.inner = false;
            for (auto& q : cs)
                if (q.inner) ++q.inner_total;
            if (!push(&CaseSolve::inner)) break;
            rho_apply_A_dot(m, m->p32, m->q32, S_PQ);
            k32_cg_update(m, n, m->e32, r32, m->p32, m->q32, S_RR);
            readback_batch(m, bs->mir_d);
            for (int i = 0; i < nc; ++i) {
                CaseSolve& q = cs[i];
                if (!q.inner || q.err) continue;
                if (S(i, S_ERR) != 0.0) {
                    fail(i, VOF_ERR_TIMEOUT, "a bounded device wait (TMA loads or a grid barrier) gave up");
                    continue;
                }
                const double rr = S(i, S_RR);
                if (!std::isfinite(rr)) {
                    fail(i, VOF_ERR_NONFINITE, "non-finite inner residual");
                    continue;
                }
                if (rr <= q.tol_in * q.tol_in * q.rr0) q.inner = false;
            }
            if (!push(&CaseSolve::inner)) break;
            run_vcycle<float>(m);
            krylov_dots(m, n, z32, r32, m->q32);
            k32_p_update(m, n, m->p32, z32);
        }
        if (!push(&CaseSolve::outer)) break;
        // FP64 update and true residual
        k32_add_to_f64(m, n, m->e32, m->p);
        launch_residual_to32(m, m->p, m->b, r32, S_RR);
        readback_batch(m, bs->mir_d);
        for (int i = 0; i < nc; ++i) {
            CaseSolve& q = cs[i];
            if (!q.outer || q.err) continue;
            q.res = std::sqrt(S(i, S_RR)) / q.bnorm;
            if (S(i, S_ERR) != 0.0) {
                fail(i, VOF_ERR_TIMEOUT, "a bounded device wait (TMA loads or a grid barrier) gave up");
                continue;
            }
            if (!std::isfinite(q.res)) {
                fail(i, VOF_ERR_NONFINITE, "non-finite residual");
                continue;
            }
            ++q.outer_n;
            q.conv = q.res <= rtol;
            if (q.conv) q.outer = false;
        }
    }
    const vof_status cst = cuda_check(m, cudaGetLastError(), "batched pressure solve");
    m->bat_n = 1;
    m->bat_stride = 0;
    m->bat_act = nullptr;
    // the rest of each case's solve on its own stream: P = 0 for a zero right
    // side, else P made mean-free
    for (int i = 0; i < nc; ++i) {
        if (!run[i]) continue;
        vof_ctx* c = cases[i];
        if (cst != VOF_OK) {
            status[i] = cst;
            continue;
        }
        if (cs[i].err) continue;
        if (cs[i].zero) {
            launch_zero(c, c->p, n);
            continue;
        }
        launch_sub_mean(c, c->p, n, S_SUM);
        reps[i].iters = cs[i].inner_total;
        reps[i].refinements = cs[i].outer_n;
        reps[i].res0 = cs[i].res0;
        reps[i].res = cs[i].res;
        if (!cs[i].conv)
            status[i] = set_err(c, VOF_ERR_NOT_CONVERGED,
                                "pressure solve did not reach rtol within max_iter (res=" +
                                    std::to_string(cs[i].res) + ")");
    }
    return cst;
}

// ---------------------------------------------------------------------------
// The batched solve captured whole. The host loop of solve_mixed_batch takes
// its per-case decisions after readbacks; here one thread per case takes the
// same decisions on the device (those of the single duct's captured solve,
// k_ctl_*), keeps each case's loop flags in its scalars (S_OUTACT, S_INACT),
// writes the flags the batched kernels read (act) and sets the WHILE handles
// while any case goes on. The kernels and their order per case are those of
// the host loop, so the iterates are the same bits.
// ---------------------------------------------------------------------------
namespace {

struct BatchCtl {
    double* scal0;      // case 0's scalars; case i's are stride bytes further
    long long stride;
    int* act;
    int nc;
    SolveCtl p;
    long long* trips;   // passes of the outer and inner loop bodies
};

__device__ __forceinline__ double* case_scal(const BatchCtl& b, int i) {
    return (double*)((char*)b.scal0 + (long long)i * b.stride);
}

// every case takes part in the dense setup; the loop counters start at zero
__global__ void k_bctl_begin(BatchCtl b) {
    for (int i = threadIdx.x; i < b.nc; i += blockDim.x) b.act[i] = 1;
    if (threadIdx.x == 0) b.trips[0] = b.trips[1] = 0;
}

__global__ void k_bctl_setup(BatchCtl b, cudaGraphConditionalHandle h_out) {
    int any = 0;
    for (int i = threadIdx.x; i < b.nc; i += blockDim.x) {
        double* s = case_scal(b, i);
        const double bb = s[S_BB];
        double bnorm = sqrt(bb);
        if (!(bnorm >= 1e-300)) bnorm = 1e-300;
        const bool zero = bb == 0.0;
        const double res0 = zero ? 0.0 : sqrt(s[S_RR]) / bnorm;
        s[S_BNORM] = bnorm;
        s[S_RES0] = res0;
        s[S_RES] = res0;
        s[S_INNER] = 0.0;
        s[S_OUTER] = 0.0;
        s[S_GUARD] = 0.0;
        s[S_ZERO] = zero ? 1.0 : 0.0;
        const int status = (!zero && !isfinite(res0)) ? ST_NONFINITE : ST_OK;
        s[S_STATUS] = status;
        const bool conv = zero || res0 <= b.p.rtol;
        s[S_CONV] = conv ? 1.0 : 0.0;
        const int go = (!conv && status == ST_OK) ? 1 : 0;
        s[S_OUTACT] = go;
        s[S_INACT] = 0.0;
        b.act[i] = go;
        any |= go;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h_out, any ? 1u : 0u);
}

__global__ void k_bctl_outer_begin(BatchCtl b) {
    for (int i = threadIdx.x; i < b.nc; i += blockDim.x) {
        double* s = case_scal(b, i);
        if (s[S_OUTACT] == 0.0) continue;
        const double res = s[S_RES], bnorm = s[S_BNORM];
        const double rr0 = res * bnorm * res * bnorm;
        const double tol_in = fmax(INNER_TOL_FLOOR, 0.2 * b.p.rtol / res);
        s[S_THR] = tol_in * tol_in * rr0;
        s[S_CAP] = s[S_INNER] + b.p.cap_add;
        s[S_INACT] = 1.0;
    }
    if (threadIdx.x == 0) ++b.trips[0];
}

// after a batched CG update (S_RR of every running case formed): count the
// iteration, check the wait flag and the residual, continue while the inner
// tolerance, max_iter and the cap allow
__global__ void k_bctl_inner(BatchCtl b, cudaGraphConditionalHandle h_in, int count_pass) {
    int any = 0;
    for (int i = threadIdx.x; i < b.nc; i += blockDim.x) {
        double* s = case_scal(b, i);
        int go = 0;
        if (s[S_INACT] != 0.0) {
            const double inner = s[S_INNER] + 1.0, guard = s[S_GUARD] + 1.0;
            s[S_INNER] = inner;
            s[S_GUARD] = guard;
            int status = (int)s[S_STATUS];
            if (s[S_ERR] != 0.0) status = ST_TIMEOUT;
            const double rr = s[S_RR];
            if (status == ST_OK && !isfinite(rr)) status = ST_NONFINITE;
            s[S_STATUS] = status;
            go = (status == ST_OK && !(rr <= s[S_THR]) && inner < b.p.max_iter &&
                  inner < s[S_CAP] && guard < b.p.max_iter + 8)
                     ? 1
                     : 0;
            s[S_INACT] = go;
        }
        b.act[i] = go;
        any |= go;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        if (count_pass) ++b.trips[1];
        cudaGraphSetConditional(h_in, any ? 1u : 0u);
    }
}

// the inner loop has ended: the FP64 update and residual run for the cases
// of this refinement
__global__ void k_bctl_inner_exit(BatchCtl b) {
    for (int i = threadIdx.x; i < b.nc; i += blockDim.x)
        b.act[i] = case_scal(b, i)[S_OUTACT] != 0.0 ? 1 : 0;
}

__global__ void k_bctl_outer_end(BatchCtl b, cudaGraphConditionalHandle h_out) {
    int any = 0;
    for (int i = threadIdx.x; i < b.nc; i += blockDim.x) {
        double* s = case_scal(b, i);
        int go = 0;
        if (s[S_OUTACT] != 0.0) {
            const double res = sqrt(s[S_RR]) / s[S_BNORM];
            s[S_RES] = res;
            int status = (int)s[S_STATUS];
            if (s[S_ERR] != 0.0) status = ST_TIMEOUT;
            if (status == ST_OK && !isfinite(res)) status = ST_NONFINITE;
            s[S_STATUS] = status;
            const double outer = s[S_OUTER] + 1.0;
            s[S_OUTER] = outer;
            const bool conv = res <= b.p.rtol;
            s[S_CONV] = conv ? 1.0 : 0.0;
            go = (!conv && status == ST_OK && s[S_INNER] < b.p.max_iter && outer < 50.0 &&
                  s[S_GUARD] < b.p.max_iter + 8)
                     ? 1
                     : 0;
            s[S_OUTACT] = go;
        }
        b.act[i] = go;
        any |= go;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) cudaGraphSetConditional(h_out, any ? 1u : 0u);
}

}  // namespace

vof_status captured_case_result(vof_ctx* c, vof_report* rep) {
    const double* h = c->hbuf;
    rep->iters = (int)h[S_INNER];
    rep->refinements = (int)h[S_OUTER];
    rep->res0 = h[S_RES0];
    rep->res = h[S_RES];
    rep->b_mean = h[S_MEAN];
    const int status = (int)h[S_STATUS];
    if (status == ST_TIMEOUT)
        return set_err(c, VOF_ERR_TIMEOUT,
                       "a bounded device wait (TMA loads or a grid barrier) gave up");
    if (status == ST_NONFINITE) return set_err(c, VOF_ERR_NONFINITE, "non-finite residual");
    if (h[S_CONV] == 0.0)
        return set_err(c, VOF_ERR_NOT_CONVERGED,
                       "pressure solve did not reach rtol within max_iter (res=" +
                           std::to_string(h[S_RES]) + ")");
    return VOF_OK;
}

void batch_solve_trips(const BatchSolveState* bs, long long* outer, long long* inner) {
    *outer = bs->trips_h[0];
    *inner = bs->trips_h[1];
}

bool capture_solve_mixed_batch(vof_ctx* m, int nc, long long stride, BatchSolveState* bs,
                               long long k[3]) {
    Level& L0 = m->lv[0];
    const int n = L0.ncells;
    float* r32 = L0.ff;
    float* z32 = L0.xf;
    for (cudaStream_t& s : m->cap_st)
        if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
    cudaStream_t st0 = m->st;
    cudaGraph_t g_top = capture_graph(st0);
    if (!g_top) return false;
    m->bat_n = nc;
    m->bat_stride = stride;
    m->bat_act = bs->act_d;
    m->in_solve_capture = true;
    const int nthr = nc < 1024 ? ((nc + 31) / 32) * 32 : 1024;
    const BatchCtl b{m->scal, stride, bs->act_d, nc,
                     SolveCtl{m->sv.rtol, m->sv.max_iter, std::max(20, m->sv.max_iter / 4)},
                     bs->trips_d};
    const long long n0 = m->nlaunch;
    long long k_outer = 0, k_inner = 0;
    cudaGraphConditionalHandle h_out = 0, h_in = 0;
    bool ok = cudaGraphConditionalHandleCreate(&h_out, g_top, 0, cudaGraphCondAssignDefault) ==
              cudaSuccess;
    m->nlaunch += 2;
    k_bctl_begin<<<1, nthr, 0, st0>>>(b);
    if (m->defer_dense) mg_dense_setup<float>(m, m->lv.back());
    k_bctl_setup<<<1, nthr, 0, st0>>>(b, h_out);
    cudaGraph_t g_out = ok ? capture_while(st0, h_out) : nullptr;
    ok = ok && g_out;
    if (ok) {
        const long long m0 = m->nlaunch;
        m->st = m->cap_st[0];
        ok = cudaStreamBeginCaptureToGraph(m->st, g_out, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess &&
             cudaGraphConditionalHandleCreate(&h_in, g_out, 0, cudaGraphCondAssignDefault) ==
                 cudaSuccess;
        if (ok) {
            ++m->nlaunch;
            k_bctl_outer_begin<<<1, nthr, 0, m->st>>>(b);
            launch_zero32_bat(m, m->e32, n);
            vcycle<float>(m, 0);
            krylov_dots(m, n, z32, r32, r32);
            launch_copy32_bat(m, m->p32, z32, n);
            rho_apply_A_dot(m, m->p32, m->q32, S_PQ);
            k32_cg_update(m, n, m->e32, r32, m->p32, m->q32, S_RR);
            ++m->nlaunch;
            k_bctl_inner<<<1, nthr, 0, m->st>>>(b, h_in, 0);
            cudaGraph_t g_in = capture_while(m->st, h_in);
            ok = g_in != nullptr;
            if (ok) {
                const long long i0 = m->nlaunch;
                m->st = m->cap_st[1];
                ok = cudaStreamBeginCaptureToGraph(m->st, g_in, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (ok) {
                    vcycle<float>(m, 0);
                    krylov_dots(m, n, z32, r32, m->q32);
                    k32_p_update(m, n, m->p32, z32);
                    rho_apply_A_dot(m, m->p32, m->q32, S_PQ);
                    k32_cg_update(m, n, m->e32, r32, m->p32, m->q32, S_RR);
                    ++m->nlaunch;
                    k_bctl_inner<<<1, nthr, 0, m->st>>>(b, h_in, 1);
                    cudaGraph_t gb = nullptr;
                    ok = cudaStreamEndCapture(m->st, &gb) == cudaSuccess;
                }
                m->st = m->cap_st[0];
                k_inner = m->nlaunch - i0;
            }
            m->nlaunch += 2;
            k_bctl_inner_exit<<<1, nthr, 0, m->st>>>(b);
            k32_add_to_f64(m, n, m->e32, m->p);
            launch_residual_to32(m, m->p, m->b, r32, S_RR);
            k_bctl_outer_end<<<1, nthr, 0, m->st>>>(b, h_out);
            cudaGraph_t gb = nullptr;
            ok = (cudaStreamEndCapture(m->st, &gb) == cudaSuccess) && ok;
        }
        m->st = st0;
        k_outer = m->nlaunch - m0 - k_inner;
    }
    m->in_solve_capture = false;
    m->bat_n = 1;
    m->bat_stride = 0;
    m->bat_act = nullptr;
    k[0] = m->nlaunch - n0 - k_outer - k_inner;
    k[1] = k_outer;
    k[2] = k_inner;
    m->nlaunch = n0;
    return ok;
}
