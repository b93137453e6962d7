// Device helpers shared by the VOF, curvature and surface-force kernels.
#pragma once

#include "vof_internal.cuh"

constexpr double EPS_IF = 1e-12;  // interface cells: EPS_IF < alpha < 1 - EPS_IF

struct Geo {
    Dims d;
    int per_x, per_y;
};

// alpha with ghosts: wetted walls (alpha = 1, complete wetting of the side
// walls, Section 5) or a periodic wrap
__device__ __forceinline__ double alpha_g(const Geo& g, const double* __restrict__ a, int i, int j,
                                          int k) {
    if (i < 0 || i >= g.d.nx) {
        if (!g.per_x) return 1.0;
        i = i < 0 ? i + g.d.nx : i - g.d.nx;
    }
    if (j < 0 || j >= g.d.ny) {
        if (!g.per_y) return 1.0;
        j = j < 0 ? j + g.d.ny : j - g.d.ny;
    }
    return a[cid(g.d, i, j, wrapk(k, g.d.nz))];
}

// Interface normal from the smoothed volume fraction (Section 2, Rudman):
// minus the central difference of alpha smoothed by [1,2,1]^3/64, in cell
// units, written as one 5x3x3 difference stencil per component:
// n_x = -(1/128) sum_{b,c} w_b w_c [a(i+2) + 2a(i+1) - 2a(i-1) - a(i-2)]
__device__ __forceinline__ void smoothed_normal(const Geo& g, const double* __restrict__ a, int i,
                                                int j, int k, double n[3]) {
    const double wt[3] = {1.0, 2.0, 1.0};
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int q = -1; q <= 1; ++q)
        for (int p = -1; p <= 1; ++p) {
            const double w2 = wt[p + 1] * wt[q + 1];
            sx += w2 * (alpha_g(g, a, i + 2, j + p, k + q) + 2.0 * alpha_g(g, a, i + 1, j + p, k + q) -
                        2.0 * alpha_g(g, a, i - 1, j + p, k + q) - alpha_g(g, a, i - 2, j + p, k + q));
            sy += w2 * (alpha_g(g, a, i + p, j + 2, k + q) + 2.0 * alpha_g(g, a, i + p, j + 1, k + q) -
                        2.0 * alpha_g(g, a, i + p, j - 1, k + q) - alpha_g(g, a, i + p, j - 2, k + q));
            sz += w2 * (alpha_g(g, a, i + p, j + q, k + 2) + 2.0 * alpha_g(g, a, i + p, j + q, k + 1) -
                        2.0 * alpha_g(g, a, i + p, j + q, k - 1) - alpha_g(g, a, i + p, j + q, k - 2));
        }
    n[0] = -sx / 128.0;
    n[1] = -sy / 128.0;
    n[2] = -sz / 128.0;
}
