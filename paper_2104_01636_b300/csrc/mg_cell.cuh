// Per-cell arithmetic of the coarse multigrid levels, shared by the
// one-launch-per-operation kernels (k_mg.cu) and the one-launch coarse tail
// (k_mg_tail.cu), so both evaluate every cell with the same expressions.
// LD loads a value that the surrounding kernel may itself have written
// (x, f, the coarse correction); coefficients are read directly.
#pragma once

#include "vof_internal.cuh"

struct LdPlain {
    template <class T>
    __device__ __forceinline__ T operator()(const T* p) const { return *p; }
};
// L2 loads for values other blocks of the same launch wrote before a
// cluster barrier
struct LdL2 {
    __device__ __forceinline__ float operator()(const float* p) const { return __ldcg(p); }
    __device__ __forceinline__ double operator()(const double* p) const { return __ldcg(p); }
};

// a coefficient as the level's arithmetic type: FP32 and FP64 coefficients
// as stored, FP16 copies widened exactly to FP32
__device__ __forceinline__ float cval(float v) { return v; }
__device__ __forceinline__ double cval(double v) { return v; }
__device__ __forceinline__ float cval(__half v) { return __half2float(v); }

// Multiply and fused multiply-add rounded as written: the compiler may not
// contract or split them, so every kernel that evaluates a cell through
// these functions (whatever its thread mapping and unrolling) produces the
// same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Red-black Gauss-Seidel update of cell (i, j, k) on one level:
//   x_c = (h^2 f_c + sum_f beta_f x_nb) / sum_f beta_f,
// the sum formed as h^2 f_c followed by one fused multiply-add per face in
// the order west, east, south, north, below, above.
// Across a wall (beta = 0) the neighbour counts as 0 and is not read.
// MODE 1: x is zero (first pass from a zero guess), neighbours are not read.
// MODE 2: each neighbour is read as x + omega x_coarse(parent): the first
// pass after the coarse correction, with the prolongation folded in.
template <class T, int MODE, class LD, class CT>
__device__ __forceinline__ void rbgs_cell(const Dims& d, T h2, const CT* __restrict__ bx,
                                          const CT* __restrict__ by, const CT* __restrict__ bz,
                                          const T* __restrict__ xr, T* __restrict__ xw,
                                          const T* __restrict__ f, int i, int j, int k,
                                          const Dims& dc, const T* __restrict__ xc, T omega,
                                          LD ld) {
    const int c = cid(d, i, j, k);
    const int kp = wrapk(k + 1, d.nz), km = wrapk(k - 1, d.nz);
    const int iw = i > 0 ? i - 1 : i, ie = i < d.nx - 1 ? i + 1 : i;
    const int js = j > 0 ? j - 1 : j, jn = j < d.ny - 1 ? j + 1 : j;
    const int cw = cid(d, iw, j, k), ce = cid(d, ie, j, k);
    const int cs = cid(d, i, js, k), cn = cid(d, i, jn, k);
    const int cb = cid(d, i, j, km), ct = cid(d, i, j, kp);
    const T b0 = cval(bx[uid(d, i, j, k)]), b1 = cval(bx[uid(d, i + 1, j, k)]);
    const T b2 = cval(by[vid(d, i, j, k)]), b3 = cval(by[vid(d, i, j + 1, k)]);
    const T b4 = cval(bz[wid(d, i, j, k)]), b5 = cval(bz[wid(d, i, j, kp)]);
    const bool hw = i > 0, he = i < d.nx - 1, hs = j > 0, hn = j < d.ny - 1;
    T num = mul_rn(h2, ld(f + c));
    if (MODE == 2) {
        auto xv = [&](int cc, int ii, int jj, int kk) {
            return fma_rn(omega, ld(xc + cid(dc, ii >> 1, jj >> 1, kk >> 1)), ld(xr + cc));
        };
        num = fma_rn(b0, hw ? xv(cw, iw, j, k) : T(0), num);
        num = fma_rn(b1, he ? xv(ce, ie, j, k) : T(0), num);
        num = fma_rn(b2, hs ? xv(cs, i, js, k) : T(0), num);
        num = fma_rn(b3, hn ? xv(cn, i, jn, k) : T(0), num);
        num = fma_rn(b4, xv(cb, i, j, km), num);
        num = fma_rn(b5, xv(ct, i, j, kp), num);
    } else if (MODE == 0) {
        num = fma_rn(b0, hw ? ld(xr + cw) : T(0), num);
        num = fma_rn(b1, he ? ld(xr + ce) : T(0), num);
        num = fma_rn(b2, hs ? ld(xr + cs) : T(0), num);
        num = fma_rn(b3, hn ? ld(xr + cn) : T(0), num);
        num = fma_rn(b4, ld(xr + cb), num);
        num = fma_rn(b5, ld(xr + ct), num);
    }
    const T den = b0 + b1 + b2 + b3 + b4 + b5;
    xw[c] = den > T(0) ? num / den : T(0);
}

// Restriction of the residual to coarse cell (I, J, K): the mean of the 8
// children's residuals. The fluxes through the 12 faces inside the 2x2x2
// block cancel in the children's sum, so only the 24 faces on the block's
// boundary are formed:
//   sum_c r_c = sum_c f_c - (1/h^2) sum_{boundary f} beta_f (x_in - x_out).
template <class T, class LD>
__device__ __forceinline__ void restrict_cell(const Dims& df, T ih2f, const T* __restrict__ bx,
                                              const T* __restrict__ by, const T* __restrict__ bz,
                                              const T* __restrict__ xf,
                                              const T* __restrict__ ff, const Dims& dc,
                                              T* __restrict__ fc, int I, int J, int K, LD ld) {
    const bool xl = I > 0, xh = 2 * I + 2 < df.nx, yl = J > 0, yh = 2 * J + 2 < df.ny;
    T fs = T(0), flux = T(0);
    const int kk[2] = {2 * K, 2 * K + 1};
    const int kout[2] = {wrapk(2 * K - 1, df.nz), wrapk(2 * K + 2, df.nz)};
#pragma unroll
    for (int c3 = 0; c3 < 8; ++c3) {
        const int a = c3 & 1, b = (c3 >> 1) & 1, e = c3 >> 2;
        const int i = 2 * I + a, j = 2 * J + b, k = kk[e];
        const int c = cid(df, i, j, k);
        const T xc = ld(xf + c);
        fs += ld(ff + c);
        if (a ? xh : xl) {
            const int ci = a ? c + 1 : c - 1;
            flux += bx[uid(df, i + a, j, k)] * (xc - ld(xf + ci));
        }
        if (b ? yh : yl) {
            const int cj = b ? c + df.nx : c - df.nx;
            flux += by[vid(df, i, j + b, k)] * (xc - ld(xf + cj));
        }
        const int cz = cid(df, i, j, kout[e]);
        flux += bz[wid(df, i, j, e ? kout[1] : k)] * (xc - ld(xf + cz));
    }
    fc[cid(dc, I, J, K)] = T(0.125) * (fs - flux * ih2f);
}

// One row of the dense coarsest-level solve x = Minv f, by one warp: each
// lane sums its strided columns in T, the lanes' sums are added in FP64 by
// a fixed shuffle tree. The result is valid in lane 0.
template <class T, class FV>
__device__ __forceinline__ double dense_row(const T* __restrict__ row, FV fv, int n, int lane) {
    T acc = T(0);
#pragma unroll 8
    for (int j = lane; j < n; j += 32) acc = fma(row[j], fv(j), acc);
    double s = (double)acc;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}
