// Variable-coefficient pressure operator (Eq. 7, steps 6/11) and the FP64
// kernels of the outer flexible-CG iteration (the multigrid preconditioner
// lives in k_mg.cu).
//
//   (A x)_c = (1/h^2) sum_f beta_f (x_c - x_nb),  beta_f = 1 / rho_f,
//   rho_f = (rho_L + rho_R)/2 (linear face averaging, step 10).
//
// Walls carry beta = 0, so the stencil reads a clamped neighbour there and
// multiplies it by zero; z is periodic. The residual, the operator and the
// Krylov updates are FP64 in every precision mode.
#include <cuda_fp16.h>

#include <initializer_list>

#include "vof_internal.cuh"

namespace {

struct CellIdx {
    int i, j, k0, k1;
    bool act;
};

__device__ __forceinline__ CellIdx cell_range(const Dims& d, int kchunk) {
    CellIdx r;
    r.i = blockIdx.x * TBX + threadIdx.x;
    r.j = blockIdx.y * TBY + threadIdx.y;
    r.act = r.i < d.nx && r.j < d.ny;
    r.k0 = blockIdx.z * kchunk;
    r.k1 = min(r.k0 + kchunk, d.nz);
    return r;
}

// (A x)_c * h^2 without the 1/h^2 factor
__device__ __forceinline__ double stencil(const Dims& d, const double* __restrict__ bx,
                                          const double* __restrict__ by,
                                          const double* __restrict__ bz,
                                          const double* __restrict__ x, int i, int j, int k) {
    const int c = cid(d, i, j, k);
    const double xc = x[c];
    const int cw = i > 0 ? c - 1 : c;
    const int ce = i < d.nx - 1 ? c + 1 : c;
    const int cs = j > 0 ? c - d.nx : c;
    const int cn = j < d.ny - 1 ? c + d.nx : c;
    const int kp = wrapk(k + 1, d.nz);
    const int cb = cid(d, i, j, wrapk(k - 1, d.nz)), ct = cid(d, i, j, kp);
    double s = bx[uid(d, i, j, k)] * (xc - x[cw]);
    s += bx[uid(d, i + 1, j, k)] * (xc - x[ce]);
    s += by[vid(d, i, j, k)] * (xc - x[cs]);
    s += by[vid(d, i, j + 1, k)] * (xc - x[cn]);
    s += bz[wid(d, i, j, k)] * (xc - x[cb]);
    s += bz[wid(d, i, j, kp)] * (xc - x[ct]);
    return s;
}

// 1 / s in FP64 without a division: an FP32 reciprocal seed r (relative
// error e0 below 2^-22) refined by one third-order step r + r (e + e^2),
// e = 1 - s r, whose truncation error e0^3 < 2^-66 lies far below FP64
// rounding; one FMA fewer than two Newton steps. s is a positive normal
// number (a sum of densities).
__device__ __forceinline__ double rcp_cubic(double s) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"((float)s));
    const double r = (double)r0;
    const double e = fma(-s, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// rho = alpha rho_l + (1 - alpha) rho_g as one FMA, alpha (rho_l - rho_g) + rho_g.
// The kernel works with half densities h = rho / 2 (the same FMA on halved
// constants, exactly half of rho), so that a face coefficient
// 2 / (rho_L + rho_R) is the reciprocal of h_L + h_R with no multiply. Each
// thread marches up z and carries the half density of the cell below.
__global__ void k_beta(Dims d, const double* __restrict__ a, double rl, double rg,
                       double* __restrict__ bx, double* __restrict__ by, double* __restrict__ bz,
                       float* __restrict__ rho32, __half* __restrict__ rho16,
                       double* __restrict__ rho64, int kchunk) {
    CellIdx r = cell_range(d, kchunk);
    if (!r.act) return;
    const int i = r.i, j = r.j;
    const double dh = 0.5 * (rl - rg), gh = 0.5 * rg;
    auto half_rho = [&](int c) { return fma(a[c], dh, gh); };
    double hb = half_rho(cid(d, i, j, wrapk(r.k0 - 1, d.nz)));
    for (int k = r.k0; k < r.k1; ++k) {
        const int c = cid(d, i, j, k);
        const double hc = half_rho(c);
        // densities of the multigrid's finest level: 2 h, scaled after the
        // rounding (exact: a power of two)
        if (rho32) rho32[c] = 2.f * (float)hc;
        if (rho16) rho16[c] = __hmul(__double2half(hc), __float2half(2.f));
        if (rho64) rho64[c] = 2.0 * hc;
        // x-face i (between i-1 and i); the last thread also writes the wall face nx
        bx[uid(d, i, j, k)] = i == 0 ? 0.0 : rcp_cubic(half_rho(c - 1) + hc);
        if (i == d.nx - 1) bx[uid(d, d.nx, j, k)] = 0.0;
        by[vid(d, i, j, k)] = j == 0 ? 0.0 : rcp_cubic(half_rho(c - d.nx) + hc);
        if (j == d.ny - 1) by[vid(d, i, d.ny, k)] = 0.0;
        bz[wid(d, i, j, k)] = rcp_cubic(hb + hc);
        hb = hc;
    }
}

__global__ void k_apply_A(Dims d, double ih2, const double* __restrict__ bx,
                          const double* __restrict__ by, const double* __restrict__ bz,
                          const double* __restrict__ x, double* __restrict__ y, int kchunk) {
    CellIdx r = cell_range(d, kchunk);
    if (!r.act) return;
    for (int k = r.k0; k < r.k1; ++k)
        y[cid(d, r.i, r.j, k)] = stencil(d, bx, by, bz, x, r.i, r.j, k) * ih2;
}

// y = A x and the block partials of x.y
__global__ void k_apply_A_dot(Dims d, double ih2, const double* __restrict__ bx,
                              const double* __restrict__ by, const double* __restrict__ bz,
                              const double* __restrict__ x, double* __restrict__ y,
                              double* __restrict__ part, int kchunk) {
    CellIdx r = cell_range(d, kchunk);
    double acc = 0.0;
    if (r.act)
        for (int k = r.k0; k < r.k1; ++k) {
            const int c = cid(d, r.i, r.j, k);
            const double v = stencil(d, bx, by, bz, x, r.i, r.j, k) * ih2;
            y[c] = v;
            acc += x[c] * v;
        }
    acc = block_sum(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = acc;
}

// r = f - A x and the block partials of r.r
__global__ void k_residual(Dims d, double ih2, const double* __restrict__ bx,
                           const double* __restrict__ by, const double* __restrict__ bz,
                           const double* __restrict__ x, const double* __restrict__ f,
                           double* __restrict__ res, double* __restrict__ part, int kchunk) {
    CellIdx r = cell_range(d, kchunk);
    double acc = 0.0;
    if (r.act)
        for (int k = r.k0; k < r.k1; ++k) {
            const int c = cid(d, r.i, r.j, k);
            const double v = f[c] - stencil(d, bx, by, bz, x, r.i, r.j, k) * ih2;
            res[c] = v;
            acc += v * v;
        }
    acc = block_sum(acc);
    if (part && threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = acc;
}

// r = f - A x in FP64, stored as FP32 (the inner right side of the mixed
// solve), with block partials of the FP64 r.r
template <bool B>
__global__ void k_residual_to32(Bat t, Dims d, double ih2, const double* __restrict__ bx,
                                const double* __restrict__ by, const double* __restrict__ bz,
                                const double* __restrict__ x, const double* __restrict__ f,
                                float* __restrict__ r32, double* __restrict__ part, int kchunk) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.z, gridDim.z);
    if (bb.off) return;
    bx = bat_at<B>(t, bb.cs, bx);
    by = bat_at<B>(t, bb.cs, by);
    bz = bat_at<B>(t, bb.cs, bz);
    x = bat_at<B>(t, bb.cs, x);
    f = bat_at<B>(t, bb.cs, f);
    r32 = bat_at<B>(t, bb.cs, r32);
    part = bat_at<B>(t, bb.cs, part);
    CellIdx r = cell_range(d, kchunk);
    r.k0 = bb.b * kchunk;
    r.k1 = min(r.k0 + kchunk, d.nz);
    double acc = 0.0;
    if (r.act)
        for (int k = r.k0; k < r.k1; ++k) {
            const int c = cid(d, r.i, r.j, k);
            const double v = f[c] - stencil(d, bx, by, bz, x, r.i, r.j, k) * ih2;
            r32[c] = (float)v;
            acc += v * v;
        }
    acc = block_sum(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear_z(bb)] = acc;
}

// ---- flat vector kernels (fixed grid => deterministic partials) ----------
__global__ void k_dot(int n, const double* __restrict__ x, const double* __restrict__ y,
                      double* __restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        acc += x[c] * y[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum(int n, const double* __restrict__ x, double* __restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        acc += x[c];
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sub_scalar(int n, double* __restrict__ x, const double* __restrict__ s) {
    const double m = *s;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        x[c] -= m;
}

__global__ void k_copy(int n, double* __restrict__ dst, const double* __restrict__ src) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        dst[c] = src[c];
}

__global__ void k_zero(int n, double* __restrict__ x) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        x[c] = 0.0;
}

__global__ void k_cg_update(int n, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q,
                            const double* __restrict__ scal, double* __restrict__ part) {
    const double al = scal[S_ALPHA];
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        x[c] += al * p[c];
        const double rv = r[c] - al * q[c];
        r[c] = rv;
        acc += rv * rv;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_dot2(int n, const double* __restrict__ z, const double* __restrict__ r,
                       const double* __restrict__ q, double* __restrict__ pa,
                       double* __restrict__ pb) {
    double a = 0.0, b = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        a += z[c] * r[c];
        b += z[c] * q[c];
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = a;
        pb[blockIdx.x] = b;
    }
}

__global__ void k_p_update(int n, double* __restrict__ p, const double* __restrict__ z,
                           const double* __restrict__ scal) {
    const double be = scal[S_BETA];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        p[c] = z[c] + be * p[c];
}

// the flat kernels above with 16-byte accesses, two values per thread and
// pass (n2 = n / 2; arrays 16-byte aligned); a thread's terms are summed in
// index order
__global__ void k_dot_x2(int n2, const double2* __restrict__ x, const double2* __restrict__ y,
                         double* __restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x) {
        const double2 a = x[c], b = y[c];
        acc += a.x * b.x;
        acc += a.y * b.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sum_x2(int n2, const double2* __restrict__ x, double* __restrict__ part) {
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x) {
        const double2 a = x[c];
        acc += a.x;
        acc += a.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_sub_scalar_x2(int n2, double2* __restrict__ x, const double* __restrict__ s) {
    const double m = *s;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x) {
        double2 a = x[c];
        a.x -= m;
        a.y -= m;
        x[c] = a;
    }
}

__global__ void k_copy_x2(int n2, double2* __restrict__ dst, const double2* __restrict__ src) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x)
        dst[c] = src[c];
}

__global__ void k_cg_update_x2(int n2, double2* __restrict__ x, double2* __restrict__ r,
                               const double2* __restrict__ p, const double2* __restrict__ q,
                               const double* __restrict__ scal, double* __restrict__ part) {
    const double al = scal[S_ALPHA];
    double acc = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x) {
        const double2 pv = p[c], qv = q[c];
        double2 xv = x[c], rv = r[c];
        xv.x += al * pv.x;
        xv.y += al * pv.y;
        rv.x = rv.x - al * qv.x;
        rv.y = rv.y - al * qv.y;
        x[c] = xv;
        r[c] = rv;
        acc += rv.x * rv.x;
        acc += rv.y * rv.y;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_dot2_x2(int n2, const double2* __restrict__ z, const double2* __restrict__ r,
                          const double2* __restrict__ q, double* __restrict__ pa,
                          double* __restrict__ pb) {
    double a = 0.0, b = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x) {
        const double2 zv = z[c], rv = r[c], qv = q[c];
        a += zv.x * rv.x;
        a += zv.y * rv.y;
        b += zv.x * qv.x;
        b += zv.y * qv.y;
    }
    a = block_sum(a);
    b = block_sum(b);
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = a;
        pb[blockIdx.x] = b;
    }
}

__global__ void k_p_update_x2(int n2, double2* __restrict__ p, const double2* __restrict__ z,
                              const double* __restrict__ scal) {
    const double be = scal[S_BETA];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n2; c += gridDim.x * blockDim.x) {
        const double2 zv = z[c];
        double2 pv = p[c];
        pv.x = zv.x + be * pv.x;
        pv.y = zv.y + be * pv.y;
        p[c] = pv;
    }
}

__global__ void k_scalar_alpha(double* scal) {
    const double pq = scal[S_PQ];
    scal[S_ALPHA] = pq > 0.0 ? scal[S_RZ] / pq : 0.0;
}

__global__ void k_scalar_beta(double* scal) {
    const double pq = scal[S_PQ];
    scal[S_BETA] = pq > 0.0 ? -scal[S_ZQ] / pq : 0.0;
}

constexpr int FLAT_THREADS = 256;
inline int flat_blocks(int n) {
    int b = (n + FLAT_THREADS - 1) / FLAT_THREADS;
    if (b > 1184) b = 1184;
    if (b < 1) b = 1;
    return b;
}

}  // namespace

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
void launch_beta(vof_ctx* c, const double* alpha) {
    const Launch& L = c->Lc;
    VOF_LAUNCH(c, k_beta, L.grid, L.block, c->d, alpha, c->ph.rho_l, c->ph.rho_g, c->bx, c->by,
               c->bz, c->rho32, (__half*)c->rho16, c->rho64, L.kchunk);
}

void launch_beta_apply_raw(const vof_grid* g, const vof_phys* ph, const double* alpha,
                           const double* x, double* y, double* bx, double* by, double* bz,
                           int sm_count, cudaStream_t s) {
    const Dims d{g->nx, g->ny, g->nz};
    const Launch L = launch_cells(d.nx, d.ny, d.nz, sm_count);
    k_beta<<<L.grid, L.block, 0, s>>>(d, alpha, ph->rho_l, ph->rho_g, bx, by, bz, nullptr, nullptr,
                                      nullptr, L.kchunk);
    k_apply_A<<<L.grid, L.block, 0, s>>>(d, 1.0 / (g->h * g->h), bx, by, bz, x, y, L.kchunk);
}

void launch_apply_A(vof_ctx* c, const Level& l, const double* x, double* y) {
    VOF_LAUNCH(c, k_apply_A, l.L.grid, l.L.block, l.d, 1.0 / (l.h * l.h), l.bx, l.by, l.bz, x, y,
                                                  l.L.kchunk);
}

void launch_apply_A_dot(vof_ctx* c, const Level& l, const double* p, double* q, int slot) {
    int m = timer_begin(c, T_RESIDUAL);
    VOF_LAUNCH(c, k_apply_A_dot, l.L.grid, l.L.block, l.d, 1.0 / (l.h * l.h), l.bx, l.by, l.bz, p,
                                                      q, c->part + (size_t)slot * MAX_PARTIALS,
                                                      l.L.kchunk);
    timer_end(c, T_RESIDUAL, m);
    finalize_sum(c, slot, l.L.nblocks, slot, 1.0);
}

void launch_residual(vof_ctx* c, const Level& l, const double* x, const double* f, double* r,
                     int slot) {
    int m = timer_begin(c, T_RESIDUAL);
    VOF_LAUNCH(c, k_residual, l.L.grid, l.L.block, 
        l.d, 1.0 / (l.h * l.h), l.bx, l.by, l.bz, x, f, r,
        slot >= 0 ? c->part + (size_t)slot * MAX_PARTIALS : nullptr, l.L.kchunk);
    timer_end(c, T_RESIDUAL, m);
    if (slot >= 0) finalize_sum(c, slot, l.L.nblocks, slot, 1.0);
}

void launch_residual_to32(vof_ctx* c, const double* x, const double* f, float* r32, int slot) {
    const Level& l = c->lv[0];
    int m = timer_begin(c, T_RESIDUAL);
    dim3 g = l.L.grid;
    const Bat b = bat_of(c, g.z);
    auto kern = b.zb ? k_residual_to32<true> : k_residual_to32<false>;
    VOF_LAUNCH(c, kern, g, l.L.block, b, l.d, 1.0 / (l.h * l.h), l.bx, l.by, l.bz,
               x, f, r32, c->part + (size_t)slot * MAX_PARTIALS, l.L.kchunk);
    timer_end(c, T_RESIDUAL, m);
    finalize_sum(c, slot, l.L.nblocks, slot, 1.0);
}

// 16-byte accesses are possible: n even, every array 16-byte aligned
inline bool vec2_ok(int n, std::initializer_list<const void*> ptrs) {
    if (n % 2) return false;
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 16) return false;
    return true;
}

void launch_dot(vof_ctx* c, const double* x, const double* y, int n, int slot) {
    double* part = c->part + (size_t)slot * MAX_PARTIALS;
    const bool v2 = vec2_ok(n, {x, y});
    const int nb = flat_blocks(v2 ? n / 2 : n);
    if (v2)
        VOF_LAUNCH(c, k_dot_x2, nb, FLAT_THREADS, n / 2, (const double2*)x, (const double2*)y,
                   part);
    else
        VOF_LAUNCH(c, k_dot, nb, FLAT_THREADS, n, x, y, part);
    finalize_sum(c, slot, nb, slot, 1.0);
}

void launch_sub_mean(vof_ctx* c, double* x, int n, int slot_mean) {
    double* part = c->part + (size_t)slot_mean * MAX_PARTIALS;
    const bool v2 = vec2_ok(n, {x});
    const int nb = flat_blocks(v2 ? n / 2 : n);
    if (v2)
        VOF_LAUNCH(c, k_sum_x2, nb, FLAT_THREADS, n / 2, (const double2*)x, part);
    else
        VOF_LAUNCH(c, k_sum, nb, FLAT_THREADS, n, x, part);
    finalize_sum(c, slot_mean, nb, slot_mean, 1.0 / (double)n);
    if (v2)
        VOF_LAUNCH(c, k_sub_scalar_x2, nb, FLAT_THREADS, n / 2, (double2*)x, c->scal + slot_mean);
    else
        VOF_LAUNCH(c, k_sub_scalar, nb, FLAT_THREADS, n, x, c->scal + slot_mean);
}

void launch_copy(vof_ctx* c, double* dst, const double* src, int n) {
    if (vec2_ok(n, {dst, src}))
        VOF_LAUNCH(c, k_copy_x2, flat_blocks(n / 2), FLAT_THREADS, n / 2, (double2*)dst,
                   (const double2*)src);
    else
        VOF_LAUNCH(c, k_copy, flat_blocks(n), FLAT_THREADS, n, dst, src);
}

void launch_zero(vof_ctx* c, double* x, int n) {
    VOF_LAUNCH(c, k_zero, flat_blocks(n), FLAT_THREADS, n, x);
}

void launch_cg_update(vof_ctx* c, int n, double* x, double* r, const double* p, const double* q,
                      int slot) {
    const bool v2 = vec2_ok(n, {x, r, p, q});
    const int nb = flat_blocks(v2 ? n / 2 : n);
    int m = timer_begin(c, T_KRYLOV);
    if (v2)
        VOF_LAUNCH(c, k_cg_update_x2, nb, FLAT_THREADS, n / 2, (double2*)x, (double2*)r,
                   (const double2*)p, (const double2*)q, c->scal,
                   c->part + (size_t)slot * MAX_PARTIALS);
    else
        VOF_LAUNCH(c, k_cg_update, nb, FLAT_THREADS, n, x, r, p, q, c->scal,
                   c->part + (size_t)slot * MAX_PARTIALS);
    timer_end(c, T_KRYLOV, m);
    finalize_sum(c, slot, nb, slot, 1.0);
}

void launch_dot2(vof_ctx* c, int n, const double* z, const double* r, const double* q, int sa,
                 int sb) {
    const bool v2 = vec2_ok(n, {z, r, q});
    const int nb = flat_blocks(v2 ? n / 2 : n);
    int m = timer_begin(c, T_KRYLOV);
    if (v2)
        VOF_LAUNCH(c, k_dot2_x2, nb, FLAT_THREADS, n / 2, (const double2*)z, (const double2*)r,
                   (const double2*)q, c->part + (size_t)sa * MAX_PARTIALS,
                   c->part + (size_t)sb * MAX_PARTIALS);
    else
        VOF_LAUNCH(c, k_dot2, nb, FLAT_THREADS, n, z, r, q, c->part + (size_t)sa * MAX_PARTIALS,
                   c->part + (size_t)sb * MAX_PARTIALS);
    timer_end(c, T_KRYLOV, m);
    finalize_sum(c, sa, nb, sa, 1.0);
    finalize_sum(c, sb, nb, sb, 1.0);
}

void launch_p_update(vof_ctx* c, int n, double* p, const double* z) {
    int m = timer_begin(c, T_KRYLOV);
    if (vec2_ok(n, {p, z}))
        VOF_LAUNCH(c, k_p_update_x2, flat_blocks(n / 2), FLAT_THREADS, n / 2, (double2*)p,
                   (const double2*)z, c->scal);
    else
        VOF_LAUNCH(c, k_p_update, flat_blocks(n), FLAT_THREADS, n, p, z, c->scal);
    timer_end(c, T_KRYLOV, m);
}

void launch_scalar_alpha(vof_ctx* c) { VOF_LAUNCH(c, k_scalar_alpha, 1, 1, c->scal); }
void launch_scalar_beta(vof_ctx* c) { VOF_LAUNCH(c, k_scalar_beta, 1, 1, c->scal); }
