// Geometric VOF advection (Eq. 3; the geometric construction with a
// direction-split update, Section 2.1):
//   reconstruct: per interface cell the normal n = -grad(alpha smoothed by
//                [1,2,1]^3/64) and the FP64 plane constant d;
//   face flux:   signed liquid volume in the donor slab of width |u| dt;
// The FP64 geometry runs only for the interface cells, compacted into a list
// each sweep so that warps are not held up by the few cut cells among them.
//   update:      alpha <- alpha - (F+ - F-) + c (u+ - u-) dt/h, clipped,
//                with c = [alpha^n > 1/2] frozen over the three sweeps so
//                the volume is conserved to round-off when div u = 0.
// Each face flux is computed once and stored, so the update telescopes
// exactly.
#include "plic.cuh"
#include "vof_geom.cuh"
#include "vof_internal.cuh"

namespace {

// PLIC plane of one cell: normal (cell units) and plane constant
struct __align__(32) Plane {
    double n0, n1, n2, d;
};

// Pass 1: clear the plane flags and append the interface cells to a list
// (warp-aggregated atomic; the list order never changes any value).
__global__ void k_if_list(Dims d, const double* __restrict__ a, unsigned char* __restrict__ has,
                          int* __restrict__ list, int* __restrict__ count, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    const unsigned lane = (threadIdx.x + TBX * threadIdx.y) & 31;
    const unsigned below = (1u << lane) - 1u;
    // a warp (one row of 32 cells) takes eight planes at a time: their
    // alpha loads in flight together, and one atomic for all their
    // interface cells
    constexpr int G = 8;
    for (int kb = k0; kb < k1; kb += G) {
        unsigned m[G];
        int tot = 0;
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int k = kb + q;
            bool itf = false;
            if (act && k < k1) {
                const int c = cid(d, i, j, k);
                // eps < alpha < 1 - eps on the integer pipe: for doubles >= +0
                // the order of the bit patterns is the order of the values, and
                // a negative alpha (sign bit set) compares below eps
                const long long ab = __double_as_longlong(a[c]);
                itf = ab > __double_as_longlong(EPS_IF) && ab < __double_as_longlong(1.0 - EPS_IF);
                has[c] = 0;
            }
            m[q] = __ballot_sync(0xffffffffu, itf);
            tot += __popc(m[q]);
        }
        if (tot) {
            int base = 0;
            if (lane == 0) base = atomicAdd(count, tot);
            base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
            for (int q = 0; q < G; ++q) {
                if ((m[q] >> lane) & 1u) list[base + __popc(m[q] & below)] = cid(d, i, j, kb + q);
                base += __popc(m[q]);
            }
        }
    }
}

// Pass 2: normal and FP64 plane constant of every listed interface cell, in
// four launches so that the plane constants run in warps of one branch:
//  (a) the normal (stored in the plane) and the estimated branch of every
//      listed cell, counted per branch;
//  (b) (one block) the start of each branch's range in if_perm;
//  (c) every cell with a plane placed in its branch's range;
//  (d) the plane constant of every cell in that order.
// Each cell's normal and plane constant are the same expressions as in one
// pass, so the planes do not depend on the order.
constexpr int NPIECE = 6;
// slots of if_count (16 ints): 0 the list's length, 1-6 the counts per
// branch, 8-13 the branches' cursors in if_perm, 14 the cells with a plane
constexpr int PIECE_CNT = 1, PIECE_CUR = 8;
static_assert(PIECE_CUR + NPIECE < 16, "if_count holds 16 ints");

// 64 registers (eight blocks per SM instead of five, no spills): more warps
// hide the alpha loads of the difference stencils
__global__ void __launch_bounds__(128, 8) k_reconstruct_normals(Geo g, const double* __restrict__ a,
                                      const int* __restrict__ list, int* __restrict__ cnt,
                                      unsigned char* __restrict__ piece, Plane* __restrict__ plane) {
    __shared__ int bc[NPIECE];
    if (threadIdx.x < NPIECE) bc[threadIdx.x] = 0;
    __syncthreads();
    const int n = cnt[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int c = list[t];
        const int i = c % g.d.nx, j = (c / g.d.nx) % g.d.ny, k = c / (g.d.nx * g.d.ny);
        double nrm[3];
        smoothed_normal(g, a, i, j, k, nrm);
        unsigned char pc = 255;
        if (nrm[0] != 0.0 || nrm[1] != 0.0 || nrm[2] != 0.0) {
            Plane& pl = plane[c];
            pl.n0 = nrm[0];
            pl.n1 = nrm[1];
            pl.n2 = nrm[2];
            pc = (unsigned char)plic::plane_piece_estimate(nrm[0], nrm[1], nrm[2], a[c]);
            atomicAdd(&bc[pc], 1);
        }
        piece[t] = pc;
    }
    __syncthreads();
    if (threadIdx.x < NPIECE && bc[threadIdx.x]) atomicAdd(&cnt[PIECE_CNT + threadIdx.x], bc[threadIdx.x]);
}

__global__ void k_piece_offsets(int* __restrict__ cnt) {
    if (threadIdx.x != 0) return;
    int o = 0;
    for (int p = 0; p < NPIECE; ++p) {
        cnt[PIECE_CUR + p] = o;
        o += cnt[PIECE_CNT + p];
    }
    cnt[PIECE_CUR + NPIECE] = o;  // cells with a plane
}

__global__ void k_piece_scatter(const int* __restrict__ list, int* __restrict__ cnt,
                                const unsigned char* __restrict__ piece, int* __restrict__ perm) {
    const int n = cnt[0];
    const unsigned lane = threadIdx.x & 31, below = (1u << lane) - 1u;
    // every lane of a warp runs the same number of passes, so the ballots
    // below always have the whole warp
    const int stride = gridDim.x * blockDim.x;
    const int base0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (int w = base0; w < n; w += stride) {
        const int t = w + (int)lane;
        const int p = t < n ? (int)piece[t] : 255;
#pragma unroll
        for (int q = 0; q < NPIECE; ++q) {
            const unsigned m = __ballot_sync(0xffffffffu, p == q);
            if (!m) continue;
            int b = 0;
            if (lane == (unsigned)(__ffs(m) - 1)) b = atomicAdd(&cnt[PIECE_CUR + q], __popc(m));
            b = __shfl_sync(0xffffffffu, b, __ffs(m) - 1);
            if (p == q) perm[b + __popc(m & below)] = list[t];
        }
    }
}

__global__ void k_reconstruct_planes(const double* __restrict__ a, const int* __restrict__ cnt,
                                     const int* __restrict__ perm, unsigned char* __restrict__ has,
                                     Plane* __restrict__ plane) {
    const int n = cnt[PIECE_CUR + NPIECE];  // cells with a plane
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int c = perm[u];
        Plane& pl = plane[c];
        pl.d = plic::plane_constant(pl.n0, pl.n1, pl.n2, a[c]);
        has[c] = 1;
    }
}

// Pass 3: every face of direction dir whose donor carries no plane moves
// the donor's uniform content, F = |u| dt/h * alpha (signed); wall faces 0.
// Faces whose donor carries a plane are left to pass 4.
__global__ void k_face_flux_simple(Geo g, int dir, const double* __restrict__ a,
                                   const unsigned char* __restrict__ has,
                                   const double* __restrict__ vel, double* __restrict__ flux,
                                   double dt_h, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= g.d.nx || j >= g.d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, g.d.nz);
    const Dims& d = g.d;
    for (int k = k0; k < k1; ++k) {
        int f, cL;
        const int cR = cid(d, i, j, k);
        bool wall = false;
        if (dir == 0) {
            f = uid(d, i, j, k);
            wall = (i == 0 && !g.per_x);
            cL = cid(d, i == 0 ? d.nx - 1 : i - 1, j, k);
        } else if (dir == 1) {
            f = vid(d, i, j, k);
            wall = (j == 0 && !g.per_y);
            cL = cid(d, i, j == 0 ? d.ny - 1 : j - 1, k);
        } else {
            f = wid(d, i, j, k);
            cL = cid(d, i, j, wrapk(k - 1, d.nz));
        }
        const double u = wall ? 0.0 : vel[f];
        // sign and zero tests on the bits (integer pipe): u > 0, u == +-0
        const long long ub = __double_as_longlong(u);
        const int dn = ub > 0 ? cL : cR;
        if ((ub << 1) == 0) {
            flux[f] = 0.0;
        } else if (!has[dn]) {
            // (u dt/h) a is -(|u| dt/h a) exactly when u < 0
            flux[f] = u * dt_h * a[dn];
        }
        // the far wall (or periodic duplicate) face is never a minus face
        if (dir == 0 && i == d.nx - 1) flux[uid(d, d.nx, j, k)] = 0.0;
        if (dir == 1 && j == d.ny - 1) flux[vid(d, i, d.ny, k)] = 0.0;
    }
}

// Pass 4: the donor-slab volume through each face whose donor is a listed
// cell with a plane: its plus face when that face's velocity is positive,
// its minus face when negative.
__global__ void k_face_flux_list(Geo g, int dir, const int* __restrict__ list,
                                 const int* __restrict__ count,
                                 const unsigned char* __restrict__ has,
                                 const Plane* __restrict__ plane, const double* __restrict__ vel,
                                 double* __restrict__ flux, double dt_h) {
    const Dims& d = g.d;
    const int n = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int c = list[t];
        if (!has[c]) continue;
        const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / (d.nx * d.ny);
        int fm, fp;
        bool wm = false, wp = false;
        if (dir == 0) {
            fm = uid(d, i, j, k);
            fp = uid(d, i + 1 == d.nx && g.per_x ? 0 : i + 1, j, k);
            wm = i == 0 && !g.per_x;
            wp = i == d.nx - 1 && !g.per_x;
        } else if (dir == 1) {
            fm = vid(d, i, j, k);
            fp = vid(d, i, j + 1 == d.ny && g.per_y ? 0 : j + 1, k);
            wm = j == 0 && !g.per_y;
            wp = j == d.ny - 1 && !g.per_y;
        } else {
            fm = wid(d, i, j, k);
            fp = wid(d, i, j, wrapk(k + 1, d.nz));
        }
        const Plane pl = plane[c];
        if (!wp) {
            const double u = vel[fp];
            if (u > 0.0)
                flux[fp] = plic::slab_fraction(pl.n0, pl.n1, pl.n2, pl.d, dir, u * dt_h, true);
        }
        if (!wm) {
            const double u = vel[fm];
            if (u < 0.0)
                flux[fm] = -plic::slab_fraction(pl.n0, pl.n1, pl.n2, pl.d, dir, -u * dt_h, false);
        }
    }
}

__global__ void k_vof_update(Geo g, int dir, const double* __restrict__ ain,
                             double* __restrict__ aout, const double* __restrict__ flux,
                             const double* __restrict__ vel, const unsigned char* __restrict__ cm,
                             double dt_h, double* __restrict__ part, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const Dims& d = g.d;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    double clip = 0.0;
    if (act)
        for (int k = k0; k < k1; ++k) {
            const int c = cid(d, i, j, k);
            int fm, fp;
            bool wm = false, wp = false;
            if (dir == 0) {
                fm = uid(d, i, j, k);
                fp = uid(d, i + 1 == d.nx && g.per_x ? 0 : i + 1, j, k);
                wm = i == 0 && !g.per_x;
                wp = i == d.nx - 1 && !g.per_x;
            } else if (dir == 1) {
                fm = vid(d, i, j, k);
                fp = vid(d, i, j + 1 == d.ny && g.per_y ? 0 : j + 1, k);
                wm = j == 0 && !g.per_y;
                wp = j == d.ny - 1 && !g.per_y;
            } else {
                fm = wid(d, i, j, k);
                fp = wid(d, i, j, wrapk(k + 1, d.nz));
            }
            const double Fm = wm ? 0.0 : flux[fm], Fp = wp ? 0.0 : flux[fp];
            const double vm = wm ? 0.0 : vel[fm], vp = wp ? 0.0 : vel[fp];
            const double an0 = ain[c] - (Fp - Fm);
            const double an = cm[c] ? an0 + (vp - vm) * dt_h : an0;
            // clip to [0, 1] with the range tests on the bits: negative
            // (sign set), above 1 (a larger pattern than that of 1.0)
            const long long ab = __double_as_longlong(an);
            double ac = an;
            if (ab < 0) {
                ac = 0.0;
                clip += an;
            } else if (ab > 0x3FF0000000000000LL) {
                ac = 1.0;
                clip += an - 1.0;
            }
            aout[c] = ac;
        }
    clip = block_sum(clip);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = clip;
}

__global__ void k_mask_volume(Dims d, const double* __restrict__ a, unsigned char* __restrict__ cm,
                              double* __restrict__ part, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    double s = 0.0;
    if (act)
        for (int k = k0; k < k1; ++k) {
            const int c = cid(d, i, j, k);
            const double ac = a[c];
            s += ac;
            // alpha > 1/2 on the integer pipe (bit-pattern order of doubles >= +0;
            // a negative alpha has the sign bit and compares below)
            if (cm) cm[c] = __double_as_longlong(ac) > __double_as_longlong(0.5);
        }
    s = block_sum(s);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = s;
}

// max |vel| over non-wall faces only (the CFL check ignores wall-face values)
__global__ void k_cfl(Geo g, const double* __restrict__ u, const double* __restrict__ v,
                      const double* __restrict__ w, double* __restrict__ part, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const Dims& d = g.d;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    // the largest magnitude on the integer pipe: with the sign bit cleared,
    // the order of the bit patterns is the order of the values
    constexpr long long MAG = 0x7FFFFFFFFFFFFFFFLL;
    auto mag = [](double x) { return __double_as_longlong(x) & MAG; };
    long long mb = 0;
    if (act)
        for (int k = k0; k < k1; ++k) {
            if (i > 0 || g.per_x) mb = max(mb, mag(u[uid(d, i, j, k)]));
            if (j > 0 || g.per_y) mb = max(mb, mag(v[vid(d, i, j, k)]));
            mb = max(mb, mag(w[wid(d, i, j, k)]));
        }
    const double m = block_max(__longlong_as_double(mb));
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = m;
}

inline Geo geo(const vof_ctx* c) { return Geo{c->d, c->g.periodic_x, c->g.periodic_y}; }

}  // namespace

void launch_vof_mask_volume(vof_ctx* c, const double* alpha, int slot) {
    const Launch& L = c->Lc;
    VOF_LAUNCH(c, k_mask_volume, L.grid, L.block, c->d, alpha, c->cmask,
                                                 c->part + (size_t)slot * MAX_PARTIALS, L.kchunk);
}

void launch_volume(vof_ctx* c, const double* alpha, int slot) {
    const Launch& L = c->Lc;
    VOF_LAUNCH(c, k_mask_volume, L.grid, L.block, c->d, alpha, nullptr,
                                                 c->part + (size_t)slot * MAX_PARTIALS, L.kchunk);
}

void launch_reconstruct(vof_ctx* c, const double* alpha) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_ADVECT);
    cudaMemsetAsync(c->if_count, 0, 64, c->st);
    VOF_LAUNCH(c, k_if_list, L.grid, L.block, c->d, alpha, c->has, c->if_list, c->if_count,
               L.kchunk);
    VOF_LAUNCH(c, k_reconstruct_normals, c->sm_count * 16, 128, geo(c), alpha, c->if_list,
               c->if_count, c->if_piece, (Plane*)c->plane);
    VOF_LAUNCH(c, k_piece_offsets, 1, 32, c->if_count);
    VOF_LAUNCH(c, k_piece_scatter, c->sm_count * 8, 256, c->if_list, c->if_count, c->if_piece,
               c->if_perm);
    VOF_LAUNCH(c, k_reconstruct_planes, c->sm_count * 16, 128, alpha, c->if_count, c->if_perm,
               c->has, (Plane*)c->plane);
    timer_end(c, T_ADVECT, m);
}

void launch_face_flux(vof_ctx* c, int dir, const double* alpha, const double* vel, double dt,
                      double* flux) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_ADVECT);
    VOF_LAUNCH(c, k_face_flux_simple, L.grid, L.block, geo(c), dir, alpha, c->has, vel, flux,
               dt / c->g.h, L.kchunk);
    VOF_LAUNCH(c, k_face_flux_list, c->sm_count * 4, 128, geo(c), dir, c->if_list, c->if_count,
               c->has, (const Plane*)c->plane, vel, flux, dt / c->g.h);
    timer_end(c, T_ADVECT, m);
}

void launch_vof_update(vof_ctx* c, int dir, const double* ain, double* aout, const double* vel,
                       const double* flux, double dt, int slot) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_ADVECT);
    VOF_LAUNCH(c, k_vof_update, L.grid, L.block, geo(c), dir, ain, aout, flux, vel, c->cmask,
                                                dt / c->g.h, c->part + (size_t)slot * MAX_PARTIALS,
                                                L.kchunk);
    timer_end(c, T_ADVECT, m);
}

void launch_cfl(vof_ctx* c, const double* u, const double* v, const double* w, double dt,
                int slot) {
    const Launch& L = c->Lc;
    VOF_LAUNCH(c, k_cfl, L.grid, L.block, geo(c), u, v, w, c->part + (size_t)slot * MAX_PARTIALS,
                                         L.kchunk);
    finalize_max(c, slot, L.nblocks, S_CFL);
    (void)dt;
}
