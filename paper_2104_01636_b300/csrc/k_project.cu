// Projection (steps 11-12) with the surface-tension jump carried by the face
// force s (Eq. 6):
//   b_c = -div(u_hat_f)_c / dt - div(beta s)_c      (wall faces carry nothing)
//   a_f = beta_f ((P_R - P_L)/h - s_f)               (zero on wall faces)
//   u_f = u_hat_f - dt a_f,  u_c = u_hat_c - dt (a_f- + a_f+)/2 per component
#include "vof_internal.cuh"

namespace {

__global__ void k_rhs(Dims d, const double* __restrict__ u, const double* __restrict__ v,
                      const double* __restrict__ w, const double* __restrict__ bx,
                      const double* __restrict__ by, const double* __restrict__ bz,
                      const double* __restrict__ sx, const double* __restrict__ sy,
                      const double* __restrict__ sz, double cu, double cs,
                      double* __restrict__ b, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    // cs * (+0): the force term of a cell whose six face forces are all +0
    const double zs = cs * 0.0;
    for (int k = k0; k < k1; ++k) {
        const int ul = uid(d, i, j, k), uh = ul + 1;
        const int vl = vid(d, i, j, k), vh = vl + d.nx;
        const int wl = wid(d, i, j, k), wh = wid(d, i, j, wrapk(k + 1, d.nz));
        const bool wx0 = i == 0, wx1 = i == d.nx - 1, wy0 = j == 0, wy1 = j == d.ny - 1;
        const double du = (wx1 ? 0.0 : u[uh]) - (wx0 ? 0.0 : u[ul]) + (wy1 ? 0.0 : v[vh]) -
                          (wy0 ? 0.0 : v[vl]) + w[wh] - w[wl];
        const double sxh = wx1 ? 0.0 : sx[uh], sxl = wx0 ? 0.0 : sx[ul];
        const double syh = wy1 ? 0.0 : sy[vh], syl = wy0 ? 0.0 : sy[vl];
        const double szh = sz[wh], szl = sz[wl];
        // Away from the interface every face force is +0 (bit pattern 0,
        // tested on the integer pipe): each product beta * (+0) is +0 for
        // beta >= 0, so is their signed sum, and the term is exactly zs with
        // no FP64 work and no coefficient loads
        const long long any = __double_as_longlong(sxh) | __double_as_longlong(sxl) |
                              __double_as_longlong(syh) | __double_as_longlong(syl) |
                              __double_as_longlong(szh) | __double_as_longlong(szl);
        double t = zs;
        if (any != 0) {
            const double ds = (wx1 ? 0.0 : bx[uh] * sxh) - (wx0 ? 0.0 : bx[ul] * sxl) +
                              (wy1 ? 0.0 : by[vh] * syh) - (wy0 ? 0.0 : by[vl] * syl) +
                              bz[wh] * szh - bz[wl] * szl;
            t = cs * ds;
        }
        b[cid(d, i, j, k)] = fma(cu, du, t);  // cu = -1/(h dt), cs = -1/h (or 0)
    }
}

// face acceleration a_f = beta_f ((P_R - P_L)/h - s_f) (zero on walls),
// stored for the cell correction, and u_f -= dt a_f
__global__ void k_correct_faces(Dims d, const double* __restrict__ P, const double* __restrict__ bx,
                                const double* __restrict__ by, const double* __restrict__ bz,
                                const double* __restrict__ sx, const double* __restrict__ sy,
                                const double* __restrict__ sz, double dt, double inv_h,
                                double* __restrict__ u, double* __restrict__ v,
                                double* __restrict__ w, double* __restrict__ ax,
                                double* __restrict__ ay, double* __restrict__ az, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        const double pc = P[c];
        int f = uid(d, i, j, k);
        const double a0 = i == 0 ? 0.0 : bx[f] * ((pc - P[c - 1]) * inv_h - sx[f]);
        ax[f] = a0;
        u[f] = i == 0 ? 0.0 : u[f] - dt * a0;
        if (i == d.nx - 1) {
            u[f + 1] = 0.0;
            ax[f + 1] = 0.0;
        }
        f = vid(d, i, j, k);
        const double a1 = j == 0 ? 0.0 : by[f] * ((pc - P[c - d.nx]) * inv_h - sy[f]);
        ay[f] = a1;
        v[f] = j == 0 ? 0.0 : v[f] - dt * a1;
        if (j == d.ny - 1) {
            v[f + d.nx] = 0.0;
            ay[f + d.nx] = 0.0;
        }
        f = wid(d, i, j, k);
        const double a2 = bz[f] * ((pc - P[cid(d, i, j, wrapk(k - 1, d.nz))]) * inv_h - sz[f]);
        az[f] = a2;
        w[f] = w[f] - dt * a2;
    }
}

// cell correction: each component minus dt times the mean of the two face
// accelerations in its direction (f -> c averaging, step 12)
__global__ void k_correct_cells(Dims d, const double* __restrict__ uh,
                                const double* __restrict__ vh, const double* __restrict__ wh,
                                const double* __restrict__ ax, const double* __restrict__ ay,
                                const double* __restrict__ az, double dt, double* __restrict__ uc,
                                double* __restrict__ vc, double* __restrict__ wc, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        const int fu = uid(d, i, j, k), fv = vid(d, i, j, k);
        uc[c] = uh[c] - dt * 0.5 * (ax[fu] + ax[fu + 1]);
        vc[c] = vh[c] - dt * 0.5 * (ay[fv] + ay[fv + d.nx]);
        wc[c] = wh[c] - dt * 0.5 * (az[wid(d, i, j, k)] + az[wid(d, i, j, wrapk(k + 1, d.nz))]);
    }
}

__global__ void k_div_max(Dims d, const double* __restrict__ u, const double* __restrict__ v,
                          const double* __restrict__ w, double inv_h, double* __restrict__ pdiv,
                          double* __restrict__ pmax, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    // maxima of magnitudes on the integer pipe: for non-negative doubles the
    // order of the bit patterns is the order of the values
    constexpr long long MAG = 0x7FFFFFFFFFFFFFFFLL;
    auto mag = [](double x) { return __double_as_longlong(x) & MAG; };
    long long md = 0, mu = 0;
    if (act)
        for (int k = k0; k < k1; ++k) {
            const int ul = uid(d, i, j, k), vl = vid(d, i, j, k), wl = wid(d, i, j, k);
            const int wh = wid(d, i, j, wrapk(k + 1, d.nz));
            const double dv = (u[ul + 1] - u[ul] + v[vl + d.nx] - v[vl] + w[wh] - w[wl]) * inv_h;
            md = max(md, mag(dv));
            mu = max(mu, max(mag(u[ul + 1]), max(mag(v[vl + d.nx]), mag(w[wl]))));
        }
    const double mdd = block_max(__longlong_as_double(md));
    const double mud = block_max(__longlong_as_double(mu));
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        pdiv[block_linear()] = mdd;
        pmax[block_linear()] = mud;
    }
}

}  // namespace

// terms: bit 0 the velocity divergence -div(u_hat)/dt, bit 1 the surface
// force -div(beta s)
void launch_rhs(vof_ctx* c, const double* u, const double* v, const double* w, const double* sx,
                const double* sy, const double* sz, double dt, double* b, int terms) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_RHS);
    const double cu = (terms & 1) ? -1.0 / (c->g.h * dt) : 0.0;
    const double cs = (terms & 2) ? -1.0 / c->g.h : 0.0;
    VOF_LAUNCH(c, k_rhs, L.grid, L.block, c->d, u, v, w, c->bx, c->by, c->bz, sx, sy, sz, cu, cs,
               b, L.kchunk);
    timer_end(c, T_RHS, m);
}

__global__ void k_lincomb(int n, double a, const double* __restrict__ x, double b,
                          const double* __restrict__ y, double* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        out[e] = a * x[e] + b * y[e];
}

void launch_lincomb(vof_ctx* c, int n, double a, const double* x, double b, const double* y,
                    double* out) {
    VOF_LAUNCH(c, k_lincomb, 4 * c->sm_count, 256, n, a, x, b, y, out);
}

void launch_correct(vof_ctx* c, const double* P, const double* sx, const double* sy,
                    const double* sz, double dt, const double* const Uh[3], double* const Uc[3],
                    double* u, double* v, double* w, int slot_div, int slot_u) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_PROJECT);
    VOF_LAUNCH(c, k_correct_faces, L.grid, L.block, c->d, P, c->bx, c->by, c->bz, sx, sy, sz, dt,
               1.0 / c->g.h, u, v, w, c->fx, c->fy, c->fz, L.kchunk);
    VOF_LAUNCH(c, k_correct_cells, L.grid, L.block, c->d, Uh[0], Uh[1], Uh[2], c->fx, c->fy, c->fz,
               dt, Uc[0], Uc[1], Uc[2], L.kchunk);
    VOF_LAUNCH(c, k_div_max, L.grid, L.block, c->d, u, v, w, 1.0 / c->g.h,
               c->part + (size_t)slot_div * MAX_PARTIALS, c->part + (size_t)slot_u * MAX_PARTIALS,
               L.kchunk);
    timer_end(c, T_PROJECT, m);
    finalize_max(c, slot_div, L.nblocks, S_MAXDIV);
    finalize_max(c, slot_u, L.nblocks, S_MAXU);
}
