// Height-function curvature and the sharp surface force (Eq. 6; steps 5-7).
// The curvature runs only for the interface cells, compacted into a list.
//
// kappa is the divergence of the unit normal pointing into the liquid
// (a gas sphere of radius R has kappa = 2/R). At an interface cell the
// column direction is the dominant component of the smoothed normal (ties
// within a relative 1e-9 go to the lower axis), the heights are 7-cell sums
// of alpha in the 3x3 block of columns (Section 2, Cummins et al.), and with
// undivided differences H_1, H_2, H_11, H_22, H_12 of the column sums
//   kappa = [H_11 (1 + H_2^2) + H_22 (1 + H_1^2) - 2 H_12 H_1 H_2]
//           / (h (1 + H_1^2 + H_2^2)^{3/2}),
// which holds for either orientation of the column because the sums count
// liquid. A column set is valid when every column starts and ends in
// opposite phases (alpha >= 1/2 against alpha < 1/2).
//
// The face force is s_f = sigma kappa_f (G_R - G_L)/h with the gas indicator
// G = [alpha < 1/2]; kappa_f is the mean of the valid values of the two
// cells, else the mean over the valid cells of the 2x3x3 block around the
// face, else 0.
#include "vof_geom.cuh"
#include "vof_internal.cuh"

namespace {

// Pass 1: zero kappa and the validity flags of every cell and append the
// interface cells to a list (warp-aggregated atomic; the order never
// changes a value), so that the FP64 height-function work runs only for
// them, in full warps.
__global__ void k_curv_list(Dims d, const double* __restrict__ a, double* __restrict__ kappa,
                            unsigned char* __restrict__ valid, int* __restrict__ list,
                            int* __restrict__ count, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    const unsigned lane = (threadIdx.x + TBX * threadIdx.y) & 31;
    const unsigned below = (1u << lane) - 1u;
    // a warp (one row of 32 cells) takes eight planes at a time: their
    // loads in flight together, one atomic for all their interface cells
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
                // eps < alpha < 1 - eps on the integer pipe (bit-pattern order of
                // doubles >= +0; a negative alpha compares below eps)
                const long long ab = __double_as_longlong(a[c]);
                itf = ab > __double_as_longlong(EPS_IF) && ab < __double_as_longlong(1.0 - EPS_IF);
                kappa[c] = 0.0;
                valid[c] = 0;
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

// Pass 2: curvature of every listed interface cell.
__global__ void k_curvature_list(Geo g, const double* __restrict__ a,
                                 const int* __restrict__ list, const int* __restrict__ count,
                                 double* __restrict__ kappa, unsigned char* __restrict__ valid,
                                 double inv_h, int exact, double kappa_exact) {
    const int n = *count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int c = list[t];
        const int i = c % g.d.nx, j = (c / g.d.nx) % g.d.ny, k = c / (g.d.nx * g.d.ny);
        double kap = 0.0;
        unsigned char ok = 1;
        if (exact) {
            kap = kappa_exact;
        } else {
            double n3[3];
            smoothed_normal(g, a, i, j, k, n3);
            int dir = 0;
            double best = fabs(n3[0]);
            if (fabs(n3[1]) > best * (1.0 + 1e-9)) { dir = 1; best = fabs(n3[1]); }
            if (fabs(n3[2]) > best * (1.0 + 1e-9)) dir = 2;
            const int t1 = dir == 0 ? 1 : 0, t2 = dir == 2 ? 1 : 2;
            double col[3][3];
            for (int p = -1; p <= 1; ++p)
                for (int q = -1; q <= 1; ++q) {
                    double s = 0.0, lo = 0.0, hi = 0.0;
                    for (int r = -3; r <= 3; ++r) {
                        int o[3];
                        o[dir] = r;
                        o[t1] = p;
                        o[t2] = q;
                        const double v = alpha_g(g, a, i + o[0], j + o[1], k + o[2]);
                        s += v;
                        if (r == -3) lo = v;
                        if (r == 3) hi = v;
                    }
                    col[p + 1][q + 1] = s;
                    if ((lo >= 0.5) == (hi >= 0.5)) ok = 0;
                }
            const double H1 = 0.5 * (col[2][1] - col[0][1]);
            const double H2 = 0.5 * (col[1][2] - col[1][0]);
            const double H11 = col[2][1] - 2.0 * col[1][1] + col[0][1];
            const double H22 = col[1][2] - 2.0 * col[1][1] + col[1][0];
            const double H12 = 0.25 * (col[2][2] - col[2][0] - col[0][2] + col[0][0]);
            const double den = 1.0 + H1 * H1 + H2 * H2;
            if (ok)
                kap = (H11 * (1.0 + H2 * H2) + H22 * (1.0 + H1 * H1) - 2.0 * H12 * H1 * H2) * inv_h /
                      (den * sqrt(den));
        }
        kappa[c] = kap;
        valid[c] = ok;
    }
}

struct SsfArgs {
    Geo g;
    const double* a;
    const double* kappa;
    const unsigned char* valid;
    double sigma_h;  // sigma / h
    int exact;
    double kappa_exact;
};

// force on the face of direction dir whose left cell is (i,j,k) and right
// cell is one step along dir; fb counts fallback faces
__device__ double face_force(const SsfArgs& A, int dir, int i, int j, int k, int& fb) {
    const Dims& d = A.g.d;
    int r[3] = {i, j, k};
    r[dir] += 1;
    const int cL = cid(d, i, j, wrapk(k, d.nz)), cR = cid(d, r[0], r[1], wrapk(r[2], d.nz));
    // G = [alpha < 1/2] on the integer pipe: for doubles >= +0 the order of
    // the bit patterns is the order of the values, and a negative alpha (sign
    // bit set) compares below; most faces end here, with no FP64 operation
    const long long half = __double_as_longlong(0.5);
    const bool gL = __double_as_longlong(A.a[cL]) < half, gR = __double_as_longlong(A.a[cR]) < half;
    if (gL == gR) return 0.0;
    double kf;
    if (A.exact) {
        kf = A.kappa_exact;
    } else {
        const bool vL = A.valid[cL], vR = A.valid[cR];
        if (vL && vR) {
            kf = 0.5 * (A.kappa[cL] + A.kappa[cR]);
        } else if (vL) {
            kf = A.kappa[cL];
        } else if (vR) {
            kf = A.kappa[cR];
        } else {
            const int t1 = dir == 0 ? 1 : 0, t2 = dir == 2 ? 1 : 2;
            double s = 0.0;
            int cnt = 0;
            for (int side = 0; side <= 1; ++side)
                for (int p = -1; p <= 1; ++p)
                    for (int q = -1; q <= 1; ++q) {
                        int x[3] = {i, j, k};
                        x[dir] += side;
                        x[t1] += p;
                        x[t2] += q;
                        if (x[0] < 0 || x[0] >= d.nx || x[1] < 0 || x[1] >= d.ny) continue;
                        const int cc = cid(d, x[0], x[1], wrapk(x[2], d.nz));
                        if (A.valid[cc]) {
                            s += A.kappa[cc];
                            ++cnt;
                        }
                    }
            ++fb;
            kf = cnt ? s / cnt : 0.0;
        }
    }
    // (sigma / h) kappa_f (G_R - G_L), G_R - G_L = +-1: a sign, exactly
    const double f = A.sigma_h * kf;
    return gR ? f : -f;
}

__global__ void k_ssf_faces(SsfArgs A, double* __restrict__ sx, double* __restrict__ sy,
                            double* __restrict__ sz, double* __restrict__ part, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const Dims& d = A.g.d;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    int fb = 0;
    if (act)
        for (int k = k0; k < k1; ++k) {
            sx[uid(d, i, j, k)] = i == 0 ? 0.0 : face_force(A, 0, i - 1, j, k, fb);
            if (i == d.nx - 1) sx[uid(d, d.nx, j, k)] = 0.0;
            sy[vid(d, i, j, k)] = j == 0 ? 0.0 : face_force(A, 1, i, j - 1, k, fb);
            if (j == d.ny - 1) sy[vid(d, i, d.ny, k)] = 0.0;
            sz[wid(d, i, j, k)] = face_force(A, 2, i, j, k - 1, fb);
        }
    const double t = block_sum((double)fb);
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = t;
}

}  // namespace

void launch_curvature(vof_ctx* c, const double* alpha, double* kappa, unsigned char* valid) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_SSF);
    cudaMemsetAsync(c->if_count, 0, sizeof(int), c->st);
    VOF_LAUNCH(c, k_curv_list, L.grid, L.block, c->d, alpha, kappa, valid, c->if_list, c->if_count,
               L.kchunk);
    VOF_LAUNCH(c, k_curvature_list, c->sm_count * 16, 128, Geo{c->d, 0, 0}, alpha, c->if_list,
               c->if_count, kappa, valid, 1.0 / c->g.h, c->ph.kappa_mode == VOF_KAPPA_EXACT,
               c->ph.kappa_exact);
    timer_end(c, T_SSF, m);
}

void launch_ssf_faces(vof_ctx* c, const double* alpha, const double* kappa,
                      const unsigned char* valid, double* sx, double* sy, double* sz, int slot) {
    const Launch& L = c->Lc;
    SsfArgs A{Geo{c->d, 0, 0}, alpha, kappa, valid, c->ph.sigma / c->g.h,
              c->ph.kappa_mode == VOF_KAPPA_EXACT, c->ph.kappa_exact};
    int m = timer_begin(c, T_SSF);
    VOF_LAUNCH(c, k_ssf_faces, L.grid, L.block, A, sx, sy, sz, c->part + (size_t)slot * MAX_PARTIALS,
                                               L.kchunk);
    timer_end(c, T_SSF, m);
    finalize_sum(c, slot, L.nblocks, S_FALLBACK, 1.0);
}
