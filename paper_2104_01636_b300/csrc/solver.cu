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

void readback(vof_ctx* c) {
    cudaMemcpyAsync(c->hbuf, c->scal, sizeof(double) * S_NSCALARS, cudaMemcpyDeviceToHost, c->st);
    cudaStreamSynchronize(c->st);
}

// symmetric V-cycle on the level arrays of type T (x <- M f at level l)
template <class T>
void vcycle(vof_ctx* c, int l) {
    const Level& L = c->lv[l];
    if (l == (int)c->lv.size() - 1) {
        mg_coarse<T>(c, L);
        return;
    }
    mg_zero<T>(c, L);
    for (int s = 0; s < c->sv.nu_pre; ++s) {
        mg_rbgs<T>(c, L, 0);
        mg_rbgs<T>(c, L, 1);
    }
    mg_restrict<T>(c, L, c->lv[l + 1]);
    vcycle<T>(c, l + 1);
    mg_prolong<T>(c, c->lv[l + 1], L);
    for (int s = 0; s < c->sv.nu_post; ++s) {
        mg_rbgs<T>(c, L, 1);
        mg_rbgs<T>(c, L, 0);
    }
}

// z = M r (one V-cycle), in the precision the context was created with
void precondition(vof_ctx* c) {
    Level& L0 = c->lv[0];
    if (c->sv.precision == VOF_PREC_FP64) {
        L0.x = c->z;
        L0.f = c->r;
        vcycle<double>(c, 0);
    } else {
        mg_to_f32(c, c->r, L0.ff, L0.ncells);
        vcycle<float>(c, 0);
        mg_to_f64(c, L0.xf, c->z, L0.ncells);
    }
}

}  // namespace

size_t mg_workspace_bytes(const vof_grid* g, const vof_solver* sv, int* nlevels) {
    std::vector<Dims> dims = level_dims(g);
    if (nlevels) *nlevels = (int)dims.size();
    const bool mixed = sv && sv->precision == VOF_PREC_MIXED_FP32;
    const size_t elt = mixed ? sizeof(float) : sizeof(double);
    size_t b = 0;
    for (size_t l = mixed ? 0 : 1; l < dims.size(); ++l) {
        const size_t n = (size_t)dims[l].nx * dims[l].ny * dims[l].nz;
        b += faces_bytes(dims[l], elt) + 2 * n * elt;
    }
    if (sv && sv->mg_interp == VOF_MG_TRILINEAR)  // residual scratch per non-coarsest level
        for (size_t l = 0; l + 1 < dims.size(); ++l)
            b += (size_t)dims[l].nx * dims[l].ny * dims[l].nz * elt;
    const Dims& dc = dims.back();
    const size_t nc = (size_t)dc.nx * dc.ny * dc.nz;
    b += 4 * nc * sizeof(double);
    if (nc <= (size_t)DENSE_MAX) b += nc * nc * (2 * sizeof(double) + (mixed ? sizeof(float) : 0));
    return b;
}

vof_status mg_allocate(vof_ctx* c) {
    std::vector<Dims> dims = level_dims(&c->g);
    c->lv.resize(dims.size());
    const bool mixed = c->sv.precision == VOF_PREC_MIXED_FP32;
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
        void* p = nullptr;
        if (cudaMalloc(&p, elt * (nu + nv + 3 * n)) != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, VOF_ERR_OOM, "cudaMalloc multigrid level");
        }
        c->allocs.push_back(p);
        if (mixed) {
            float* q = (float*)p;
            L.bxf = q;
            L.byf = q + nu;
            L.bzf = q + nu + nv;
            L.xf = q + nu + nv + n;
            L.ff = q + nu + nv + 2 * n;
        } else {
            double* q = (double*)p;
            L.bx = q;
            L.by = q + nu;
            L.bz = q + nu + nv;
            L.x = q + nu + nv + n;
            L.f = q + nu + nv + 2 * n;
        }
    }
    if (c->sv.mg_interp == VOF_MG_TRILINEAR) {
        const size_t elt = mixed ? sizeof(float) : sizeof(double);
        for (size_t l = 0; l + 1 < c->lv.size(); ++l) {
            void* q = nullptr;
            if (cudaMalloc(&q, elt * (size_t)c->lv[l].ncells) != cudaSuccess) {
                cudaGetLastError();
                return set_err(c, VOF_ERR_OOM, "cudaMalloc multigrid residual");
            }
            c->allocs.push_back(q);
            c->lv[l].rs = q;
        }
    }
    const Level& Lc = c->lv.back();
    void* p = nullptr;
    if (cudaMalloc(&p, 4 * sizeof(double) * (size_t)Lc.ncells) != cudaSuccess)
        return set_err(c, VOF_ERR_OOM, "cudaMalloc coarse scratch");
    c->allocs.push_back(p);
    c->coarse_scratch = (double*)p;
    if (Lc.ncells <= DENSE_MAX) {
        const size_t n2 = (size_t)Lc.ncells * Lc.ncells;
        void *a = nullptr, *b = nullptr, *f = nullptr;
        if (cudaMalloc(&a, n2 * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&b, n2 * sizeof(double)) != cudaSuccess ||
            (mixed && cudaMalloc(&f, n2 * sizeof(float)) != cudaSuccess)) {
            cudaGetLastError();
            if (a) cudaFree(a);
            if (b) cudaFree(b);
            return set_err(c, VOF_ERR_OOM, "cudaMalloc dense coarse inverse");
        }
        c->allocs.push_back(a);
        c->allocs.push_back(b);
        if (f) c->allocs.push_back(f);
        c->dense_a = (double*)a;
        c->dense_b = (double*)b;
        c->dense_inv_f = (float*)f;
        c->dense_n = Lc.ncells;
        // shift: the liquid face coefficient (the smallest physical one) per face
        c->dense_shift = 1.0 / c->ph.rho_l;
    }
    return VOF_OK;
}

void mg_build_coefficients(vof_ctx* c) {
    if (c->sv.precision == VOF_PREC_FP64) {
        for (size_t l = 1; l < c->lv.size(); ++l) mg_coarsen_beta<double>(c, c->lv[l - 1], c->lv[l]);
        if (c->dense_n > 0) mg_dense_setup<double>(c, c->lv.back());
        return;
    }
    const Level& L0 = c->lv[0];
    const int nu = (L0.d.nx + 1) * L0.d.ny * L0.d.nz, nv = L0.d.nx * (L0.d.ny + 1) * L0.d.nz;
    mg_to_f32(c, c->bx, L0.bxf, nu);
    mg_to_f32(c, c->by, L0.byf, nv);
    mg_to_f32(c, c->bz, L0.bzf, L0.ncells);
    for (size_t l = 1; l < c->lv.size(); ++l) mg_coarsen_beta<float>(c, c->lv[l - 1], c->lv[l]);
    if (c->dense_n > 0) mg_dense_setup<float>(c, c->lv.back());
}

// Solves A P = b_in - mean(b_in) with the fine-level beta already built.
vof_status solve_pressure(vof_ctx* c, const double* b_in, double* P, vof_report* rep) {
    const int n = c->lv[0].ncells;
    Level& L0 = c->lv[0];
    mg_build_coefficients(c);

    launch_copy(c, c->b, b_in, n);
    launch_sub_mean(c, c->b, n, S_MEAN);
    launch_dot(c, c->b, c->b, n, S_BB);
    launch_residual(c, L0, P, c->b, c->r, S_RR);
    readback(c);
    vof_status st = cuda_check(c, cudaGetLastError(), "pressure solve setup");
    if (st != VOF_OK) return st;
    const double b_mean = c->hbuf[S_MEAN];
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
