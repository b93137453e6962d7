// Geometric multigrid preconditioner of the pressure solve (the paper's
// multigrid-accelerated red-black relaxation, Section 2.1, used here as one
// symmetric V-cycle per Krylov iteration), templated on the scalar type:
// T = double for the FP64 path, T = float for the mixed-precision path
// (FP32 V-cycle inside the FP64 flexible-CG iteration).
//
// Level l has spacing 2^l h and halves every dimension. A coarse face
// coefficient is the mean of the four fine faces it covers (walls stay 0),
// restriction averages the fine residual over the eight children and
// prolongation adds the coarse value to its eight children; the smoother is
// red-black Gauss-Seidel, x_c = (h^2 f_c + sum beta x_nb) / sum beta. The
// coarsest level (up to DENSE_MAX cells) is solved exactly with an explicit
// inverse formed once per solve by FP64 Gauss-Jordan elimination; larger
// coarsest levels fall back to Jacobi-preconditioned CG in one thread block.
#include <algorithm>
#include <initializer_list>
#include <mutex>
#include <vector>

#include "mg_cell.cuh"
#include "vof_internal.cuh"

namespace {

template <class T>
__device__ __forceinline__ T stencil_t(const Dims& d, const T* __restrict__ bx,
                                       const T* __restrict__ by, const T* __restrict__ bz,
                                       const T* __restrict__ x, int i, int j, int k) {
    const int c = cid(d, i, j, k);
    const T xc = x[c];
    const int cw = i > 0 ? c - 1 : c;
    const int ce = i < d.nx - 1 ? c + 1 : c;
    const int cs = j > 0 ? c - d.nx : c;
    const int cn = j < d.ny - 1 ? c + d.nx : c;
    const int kp = wrapk(k + 1, d.nz);
    const int cb = cid(d, i, j, wrapk(k - 1, d.nz)), ct = cid(d, i, j, kp);
    T s = bx[uid(d, i, j, k)] * (xc - x[cw]);
    s += bx[uid(d, i + 1, j, k)] * (xc - x[ce]);
    s += by[vid(d, i, j, k)] * (xc - x[cs]);
    s += by[vid(d, i, j + 1, k)] * (xc - x[cn]);
    s += bz[wid(d, i, j, k)] * (xc - x[cb]);
    s += bz[wid(d, i, j, kp)] * (xc - x[ct]);
    return s;
}

template <class T>
__global__ void k_rbgs_t(Dims d, T h2, const T* __restrict__ bx, const T* __restrict__ by,
                         const T* __restrict__ bz, T* __restrict__ x, const T* __restrict__ f,
                         int color, int kchunk) {
    pdl_wait();
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        if (((i + j + k) & 1) != color) continue;
        const int c = cid(d, i, j, k);
        const int cw = i > 0 ? c - 1 : c;
        const int ce = i < d.nx - 1 ? c + 1 : c;
        const int cs = j > 0 ? c - d.nx : c;
        const int cn = j < d.ny - 1 ? c + d.nx : c;
        const int kp = wrapk(k + 1, d.nz);
        const int cb = cid(d, i, j, wrapk(k - 1, d.nz)), ct = cid(d, i, j, kp);
        const T b0 = bx[uid(d, i, j, k)], b1 = bx[uid(d, i + 1, j, k)];
        const T b2 = by[vid(d, i, j, k)], b3 = by[vid(d, i, j + 1, k)];
        const T b4 = bz[wid(d, i, j, k)], b5 = bz[wid(d, i, j, kp)];
        const T num = h2 * f[c] + b0 * x[cw] + b1 * x[ce] + b2 * x[cs] + b3 * x[cn] + b4 * x[cb] +
                      b5 * x[ct];
        const T den = b0 + b1 + b2 + b3 + b4 + b5;
        x[c] = den > T(0) ? num / den : T(0);
    }
}

// Same sweep with one thread per x-pair (2t, 2t+1): exactly one member has
// the sweep's colour on every plane, so no lane idles. Within one colour the
// cells written and the cells read (their neighbours, of the other colour)
// are disjoint, so x is read and written through separate restrict
// pointers to the same array, which lets loads of later planes be issued
// early. Needs an even nx (every smoothed level has one).
// MODE 1: the first pass from a zero x (the neighbours count as zero, so
// no separate zeroing pass is needed). MODE 2: the first pass after the
// coarse-grid correction, which reads each neighbour as x + omega x_coarse
// of its parent: Gauss-Seidel never reads a cell's own old value, and this
// pass and the next overwrite every cell, so no separate prolongation pass
// is needed.
// CT is the coefficients' storage type (T, or FP16 copies on a large coarse
// level of the FP32 cycle).
// FLAT: a thread per (x-pair, y, z) in 1-D blocks, the case along grid y
// (the levels with small planes, where the 32 x 8 tiles leave most lanes
// idle); the cells and their arithmetic are the same either way
template <class T, int MODE, class CT, bool B, bool FLAT = false>
__global__ void k_rbgs_pair_t(Bat bt, Dims d, T h2, const CT* __restrict__ bx,
                              const CT* __restrict__ by, const CT* __restrict__ bz,
                              const T* __restrict__ xr, T* __restrict__ xw,
                              const T* __restrict__ f, int color, int kchunk, Dims dc,
                              const T* __restrict__ xc, T omega) {
    pdl_wait();
    const BatBlk bb = bat_blk<B>(bt, FLAT ? blockIdx.y : blockIdx.z, FLAT ? gridDim.y : gridDim.z);
    if (bb.off) return;
    bx = bat_at<B>(bt, bb.cs, bx);
    by = bat_at<B>(bt, bb.cs, by);
    bz = bat_at<B>(bt, bb.cs, bz);
    xr = bat_at<B>(bt, bb.cs, xr);
    xw = bat_at<B>(bt, bb.cs, xw);
    f = bat_at<B>(bt, bb.cs, f);
    if (xc) xc = bat_at<B>(bt, bb.cs, xc);
    if (FLAT) {  // a thread per (x-pair, y, z) of the level
        const int hp = d.nx >> 1;
        const int q = blockIdx.x * blockDim.x + threadIdx.x;
        if (q >= hp * d.ny * d.nz) return;
        const int t = q % hp, r = q / hp, j = r % d.ny, k = r / d.ny;
        rbgs_cell<T, MODE>(d, h2, bx, by, bz, xr, xw, f, 2 * t + ((j + k + color) & 1), j, k, dc,
                           xc, omega, LdPlain());
        return;
    }
    const int t = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (t >= (d.nx >> 1) || j >= d.ny) return;
    const int k0 = bb.b * kchunk, k1 = min(k0 + kchunk, d.nz);
#pragma unroll 2
    for (int k = k0; k < k1; ++k)
        rbgs_cell<T, MODE>(d, h2, bx, by, bz, xr, xw, f, 2 * t + ((j + k + color) & 1), j, k, dc,
                           xc, omega, LdPlain());
}

// Restriction of the residual averaged over the 8 children (restrict_cell).
template <class T>
__global__ void k_restrict_t(Dims df, T ih2f, const T* __restrict__ bx, const T* __restrict__ by,
                             const T* __restrict__ bz, const T* __restrict__ xf,
                             const T* __restrict__ ff, Dims dc, T* __restrict__ fc, int kchunk) {
    pdl_wait();
    const int I = blockIdx.x * TBX + threadIdx.x, J = blockIdx.y * TBY + threadIdx.y;
    if (I >= dc.nx || J >= dc.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, dc.nz);
    for (int K = k0; K < k1; ++K)
        restrict_cell(df, ih2f, bx, by, bz, xf, ff, dc, fc, I, J, K, LdPlain());
}

// two adjacent coefficients (even index) as FP32
__device__ __forceinline__ float2 cpair(const float* a, int c) {
    return *reinterpret_cast<const float2*>(a + c);
}
__device__ __forceinline__ float2 cpair(const __half* a, int c) {
    return __half22float2(*reinterpret_cast<const __half2*>(a + c));
}

// restrict_cell in FP32 with the children of a row loaded as pairs: the
// two children of a row (2I, 2I+1) are adjacent, and so are their right
// sides, their y and z faces and their neighbours across in y and z
// (8-byte loads; 2I and nx are even). Same terms in the same order.
// CT: FP32 coefficients, or the level's FP16 copies (the colour passes of
// the same level read the same copies, so the cycle keeps one operator).
// FLAT: a thread per coarse cell in 1-D blocks, the case along grid y
template <class CT, bool B, bool FLAT = false>
__global__ void k_restrict_pair_f(Bat bt, Dims df, float ih2f, const CT* __restrict__ bx,
                                  const CT* __restrict__ by, const CT* __restrict__ bz,
                                  const float* __restrict__ xf, const float* __restrict__ ff,
                                  Dims dc, float* __restrict__ fc, int kchunk) {
    pdl_wait();
    const BatBlk bb = bat_blk<B>(bt, FLAT ? blockIdx.y : blockIdx.z, FLAT ? gridDim.y : gridDim.z);
    if (bb.off) return;
    bx = bat_at<B>(bt, bb.cs, bx);
    by = bat_at<B>(bt, bb.cs, by);
    bz = bat_at<B>(bt, bb.cs, bz);
    xf = bat_at<B>(bt, bb.cs, xf);
    ff = bat_at<B>(bt, bb.cs, ff);
    fc = bat_at<B>(bt, bb.cs, fc);
    int I, J, k0, k1;
    if (FLAT) {
        const int q = blockIdx.x * blockDim.x + threadIdx.x;
        if (q >= dc.nx * dc.ny * dc.nz) return;
        I = q % dc.nx;
        J = (q / dc.nx) % dc.ny;
        k0 = q / (dc.nx * dc.ny);
        k1 = k0 + 1;
    } else {
        I = blockIdx.x * TBX + threadIdx.x;
        J = blockIdx.y * TBY + threadIdx.y;
        if (I >= dc.nx || J >= dc.ny) return;
        k0 = bb.b * kchunk;
        k1 = min(k0 + kchunk, dc.nz);
    }
    const bool xl = I > 0, xh = 2 * I + 2 < df.nx, yl = J > 0, yh = 2 * J + 2 < df.ny;
    auto ld2 = [](const float* a, int c) { return *reinterpret_cast<const float2*>(a + c); };
    auto cp2 = [](const CT* a, int c) { return cpair(a, c); };
    for (int K = k0; K < k1; ++K) {
        float fs = 0.f, flux = 0.f;
        const int kk[2] = {2 * K, 2 * K + 1};
        const int kout[2] = {wrapk(2 * K - 1, df.nz), wrapk(2 * K + 2, df.nz)};
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int j = 2 * J + b, k = kk[e];
                const int c = cid(df, 2 * I, j, k);
                const float2 xc = ld2(xf, c), f2 = ld2(ff, c);
                const bool hy = b ? yh : yl;
                const float2 byf = cp2(by, vid(df, 2 * I, j + b, k));
                const float2 xy = hy ? ld2(xf, b ? c + df.nx : c - df.nx) : make_float2(0.f, 0.f);
                const float2 bzf = cp2(bz, wid(df, 2 * I, j, e ? kout[1] : k));
                const float2 xz = ld2(xf, cid(df, 2 * I, j, kout[e]));
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float xv = a ? xc.y : xc.x;
                    fs += a ? f2.y : f2.x;
                    if (a ? xh : xl)
                        flux += cval(bx[uid(df, 2 * I + a + a, j, k)]) * (xv - xf[a ? c + 2 : c - 1]);
                    if (hy) flux += (a ? byf.y : byf.x) * (xv - (a ? xy.y : xy.x));
                    flux += (a ? bzf.y : bzf.x) * (xv - (a ? xz.y : xz.x));
                }
            }
        fc[cid(dc, I, J, K)] = 0.125f * (fs - flux * ih2f);
    }
}

template <class T>
__global__ void k_prolong_t(Dims dc, const T* __restrict__ xc, Dims df, T* __restrict__ xf,
                            T omega, int kchunk) {
    pdl_wait();
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= df.nx || j >= df.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, df.nz);
    for (int k = k0; k < k1; ++k)
        xf[cid(df, i, j, k)] += omega * xc[cid(dc, i >> 1, j >> 1, k >> 1)];
}

// The same for a fine level with an even nx: a thread adds the correction
// of parent I to the fine pair (2I, 2I+1) with one 8-byte load and store.
template <bool B>
__global__ void k_prolong_pair_f(Bat bt, Dims dc, const float* __restrict__ xc, Dims df,
                                 float* __restrict__ xf, float omega, int kchunk) {
    pdl_wait();
    const BatBlk bb = bat_blk<B>(bt, blockIdx.z, gridDim.z);
    if (bb.off) return;
    xc = bat_at<B>(bt, bb.cs, xc);
    xf = bat_at<B>(bt, bb.cs, xf);
    const int I = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (2 * I >= df.nx || j >= df.ny) return;
    const int k0 = bb.b * kchunk, k1 = min(k0 + kchunk, df.nz);
    auto one = [&](int k) {
        const float cv = xc[cid(dc, I, j >> 1, k >> 1)];
        float2* p = reinterpret_cast<float2*>(xf + cid(df, 2 * I, j, k));
        float2 v = *p;
        v.x += omega * cv;
        v.y += omega * cv;
        *p = v;
    };
    int k = k0;
    if (k < k1 && (k & 1)) one(k++);
    // four planes (two parents) per pass: every load issued before the
    // stores, so a thread has four planes in flight instead of one
    for (; k + 3 < k1; k += 4) {
        const float c0 = xc[cid(dc, I, j >> 1, k >> 1)], c1 = xc[cid(dc, I, j >> 1, (k >> 1) + 1)];
        float2* p = reinterpret_cast<float2*>(xf + cid(df, 2 * I, j, k));
        const size_t pl = (size_t)df.nx * df.ny / 2;  // plane stride in pairs
        float2 v0 = p[0], v1 = p[pl], v2 = p[2 * pl], v3 = p[3 * pl];
        v0.x += omega * c0;
        v0.y += omega * c0;
        v1.x += omega * c0;
        v1.y += omega * c0;
        v2.x += omega * c1;
        v2.y += omega * c1;
        v3.x += omega * c1;
        v3.y += omega * c1;
        p[0] = v0;
        p[pl] = v1;
        p[2 * pl] = v2;
        p[3 * pl] = v3;
    }
    for (; k < k1; ++k) one(k);
}

// Cell-centred trilinear prolongation along one axis: the fine cell 2I
// takes 3/4 of coarse I and 1/4 of I-1, the fine cell 2I+1 3/4 of I and 1/4
// of I+1; across a wall the outside share goes to the parent (constant
// extension), on the periodic axis it wraps.
struct Tri {
    int lo, hi;   // the two coarse indices
    float wlo, whi;
};
__device__ __forceinline__ Tri tri1(int i, int N, bool periodic) {
    const int I = i >> 1;
    int nb = (i & 1) ? I + 1 : I - 1;
    Tri t;
    if (nb < 0 || nb >= N) {
        if (periodic) {
            nb = nb < 0 ? nb + N : nb - N;
        } else {
            t.lo = I; t.hi = I; t.wlo = 1.f; t.whi = 0.f;
            return t;
        }
    }
    t.lo = I; t.hi = nb; t.wlo = 0.75f; t.whi = 0.25f;
    return t;
}

template <class T>
__global__ void k_prolong_tri_t(Dims dc, const T* __restrict__ xc, Dims df, T* __restrict__ xf,
                                T omega, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= df.nx || j >= df.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, df.nz);
    const Tri tx = tri1(i, dc.nx, false), ty = tri1(j, dc.ny, false);
    for (int k = k0; k < k1; ++k) {
        const Tri tz = tri1(k, dc.nz, true);
        const int xs[2] = {tx.lo, tx.hi}, ys[2] = {ty.lo, ty.hi}, zs[2] = {tz.lo, tz.hi};
        const T wx[2] = {(T)tx.wlo, (T)tx.whi}, wy[2] = {(T)ty.wlo, (T)ty.whi},
                wz[2] = {(T)tz.wlo, (T)tz.whi};
        T s = T(0);
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a)
                    s += wx[a] * wy[b] * wz[c] * xc[cid(dc, xs[a], ys[b], zs[c])];
        xf[cid(df, i, j, k)] += omega * s;
    }
}

// r = f - A x on one level (the MG residual before full-weighting restriction)
template <class T>
__global__ void k_mg_residual_t(Dims d, T ih2, const T* __restrict__ bx, const T* __restrict__ by,
                                const T* __restrict__ bz, const T* __restrict__ x,
                                const T* __restrict__ f, T* __restrict__ r, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        r[c] = f[c] - stencil_t(d, bx, by, bz, x, i, j, k) * ih2;
    }
}

// weight that fine index i gives coarse index C along an axis
__device__ __forceinline__ float w1(int i, int C, int N, bool periodic) {
    const Tri t = tri1(i, N, periodic);
    float w = 0.f;
    if (t.lo == C) w += t.wlo;
    if (t.hi == C) w += t.whi;
    return w;
}

// Restriction as the transpose of the trilinear prolongation, divided by 8:
// coarse I gathers fine cells 2I-1 .. 2I+2 along each axis with the weights
// those fine cells give I when prolongating.
template <class T>
__global__ void k_restrict_fw_t(Dims df, const T* __restrict__ rf, Dims dc, T* __restrict__ fc,
                                int kchunk) {
    const int I = blockIdx.x * TBX + threadIdx.x, J = blockIdx.y * TBY + threadIdx.y;
    if (I >= dc.nx || J >= dc.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, dc.nz);
    for (int K = k0; K < k1; ++K) {
        T s = T(0);
        for (int c = -1; c <= 2; ++c) {
            int k = 2 * K + c;
            k = k < 0 ? k + df.nz : (k >= df.nz ? k - df.nz : k);
            const float wz = w1(k, K, dc.nz, true);
            if (wz == 0.f) continue;
            for (int b = -1; b <= 2; ++b) {
                const int j = 2 * J + b;
                if (j < 0 || j >= df.ny) continue;
                const float wy = w1(j, J, dc.ny, false);
                if (wy == 0.f) continue;
                for (int a = -1; a <= 2; ++a) {
                    const int i = 2 * I + a;
                    if (i < 0 || i >= df.nx) continue;
                    const float wx = w1(i, I, dc.nx, false);
                    if (wx == 0.f) continue;
                    s += (T)(wx * wy * wz) * rf[cid(df, i, j, k)];
                }
            }
        }
        fc[cid(dc, I, J, K)] = T(0.125) * s;
    }
}

template <class T, class TI = T>
__global__ void k_coarsen_beta_t(Dims df, const TI* __restrict__ bxf, const TI* __restrict__ byf,
                                 const TI* __restrict__ bzf, Dims dc, T* __restrict__ bxc,
                                 T* __restrict__ byc, T* __restrict__ bzc, int kchunk) {
    const int I = blockIdx.x * TBX + threadIdx.x, J = blockIdx.y * TBY + threadIdx.y;
    if (I >= dc.nx || J >= dc.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, dc.nz);
    for (int K = k0; K < k1; ++K) {
        const int i = 2 * I, j = 2 * J, k = 2 * K;
        bxc[uid(dc, I, J, K)] = T(TI(0.25) * (bxf[uid(df, i, j, k)] + bxf[uid(df, i, j + 1, k)] +
                                              bxf[uid(df, i, j, k + 1)] + bxf[uid(df, i, j + 1, k + 1)]));
        if (I == dc.nx - 1) bxc[uid(dc, dc.nx, J, K)] = T(0);
        byc[vid(dc, I, J, K)] = T(TI(0.25) * (byf[vid(df, i, j, k)] + byf[vid(df, i + 1, j, k)] +
                                              byf[vid(df, i, j, k + 1)] + byf[vid(df, i + 1, j, k + 1)]));
        if (J == dc.ny - 1) byc[vid(dc, I, dc.ny, K)] = T(0);
        bzc[wid(dc, I, J, K)] = T(TI(0.25) * (bzf[wid(df, i, j, k)] + bzf[wid(df, i + 1, j, k)] +
                                              bzf[wid(df, i, j + 1, k)] + bzf[wid(df, i + 1, j + 1, k)]));
    }
}

// density coarsening: a coarse cell's density is the mean of its eight
// children's; coarse faces then follow the fine-grid rule 1 / mean(rho)
template <class T>
__global__ void k_avg8_t(Dims df, const T* __restrict__ rf, Dims dc, T* __restrict__ rc,
                         int kchunk) {
    const int I = blockIdx.x * TBX + threadIdx.x, J = blockIdx.y * TBY + threadIdx.y;
    if (I >= dc.nx || J >= dc.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, dc.nz);
    for (int K = k0; K < k1; ++K) {
        T s = T(0);
        for (int c3 = 0; c3 < 8; ++c3)
            s += rf[cid(df, 2 * I + (c3 & 1), 2 * J + ((c3 >> 1) & 1), 2 * K + (c3 >> 2))];
        rc[cid(dc, I, J, K)] = T(0.125) * s;
    }
}

template <class T>
__global__ void k_beta_from_rho_t(Dims d, const T* __restrict__ rho, T* __restrict__ bx,
                                  T* __restrict__ by, T* __restrict__ bz, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        const T r = rho[c];
        bx[uid(d, i, j, k)] = i == 0 ? T(0) : T(2) / (rho[c - 1] + r);
        if (i == d.nx - 1) bx[uid(d, d.nx, j, k)] = T(0);
        by[vid(d, i, j, k)] = j == 0 ? T(0) : T(2) / (rho[c - d.nx] + r);
        if (j == d.ny - 1) by[vid(d, i, d.ny, k)] = T(0);
        bz[wid(d, i, j, k)] = T(2) / (rho[cid(d, i, j, wrapk(k - 1, d.nz))] + r);
    }
}

// Jacobi-preconditioned CG on the coarsest level, one thread block; vectors
// in T, reductions in FP64. Bounded iteration count; the result is made
// mean-free (the operator's null space is the constants).
template <class T>
__global__ void k_coarse_cg_t(Dims d, T ih2, const T* __restrict__ bx, const T* __restrict__ by,
                              const T* __restrict__ bz, const T* __restrict__ f,
                              T* __restrict__ x, T* __restrict__ scratch, int maxit, double tol) {
    __shared__ double bc[2];
    const int n = d.nx * d.ny * d.nz;
    T* rr = scratch;
    T* pp = scratch + n;
    T* qq = scratch + 2 * n;
    T* dinv = scratch + 3 * n;
    const int tid = threadIdx.x, nt = blockDim.x;
    double s = 0.0;
    for (int c = tid; c < n; c += nt) {
        const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / (d.nx * d.ny);
        const T dg = bx[uid(d, i, j, k)] + bx[uid(d, i + 1, j, k)] + by[vid(d, i, j, k)] +
                     by[vid(d, i, j + 1, k)] + bz[wid(d, i, j, k)] +
                     bz[wid(d, i, j, wrapk(k + 1, d.nz))];
        dinv[c] = dg > T(0) ? T(1) / (dg * ih2) : T(0);
        x[c] = T(0);
        rr[c] = f[c];
        s += (double)f[c];
    }
    s = block_sum(s);
    if (tid == 0) bc[0] = s / n;
    __syncthreads();
    const T fm = (T)bc[0];
    double rz = 0.0, r2 = 0.0;
    for (int c = tid; c < n; c += nt) {
        rr[c] -= fm;
        pp[c] = dinv[c] * rr[c];
        rz += (double)rr[c] * (double)pp[c];
        r2 += (double)rr[c] * (double)rr[c];
    }
    rz = block_sum(rz);
    r2 = block_sum(r2);
    if (tid == 0) { bc[0] = rz; bc[1] = r2; }
    __syncthreads();
    rz = bc[0];
    const double r20 = bc[1];
    if (r20 > 0.0) {
        for (int it = 0; it < maxit; ++it) {
            double pq = 0.0;
            for (int c = tid; c < n; c += nt) {
                const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / (d.nx * d.ny);
                const T v = stencil_t(d, bx, by, bz, pp, i, j, k) * ih2;
                qq[c] = v;
                pq += (double)pp[c] * (double)v;
            }
            pq = block_sum(pq);
            if (tid == 0) bc[0] = pq;
            __syncthreads();
            pq = bc[0];
            if (!(pq > 0.0)) break;
            const T al = (T)(rz / pq);
            double r2n = 0.0, rzn = 0.0;
            for (int c = tid; c < n; c += nt) {
                x[c] += al * pp[c];
                rr[c] -= al * qq[c];
                r2n += (double)rr[c] * (double)rr[c];
                rzn += (double)rr[c] * (double)dinv[c] * (double)rr[c];
            }
            r2n = block_sum(r2n);
            rzn = block_sum(rzn);
            if (tid == 0) { bc[0] = r2n; bc[1] = rzn; }
            __syncthreads();
            r2n = bc[0];
            rzn = bc[1];
            if (r2n <= tol * tol * r20) break;
            const T be = (T)(rzn / rz);
            rz = rzn;
            for (int c = tid; c < n; c += nt) pp[c] = dinv[c] * rr[c] + be * pp[c];
            __syncthreads();
        }
    }
    s = 0.0;
    for (int c = tid; c < n; c += nt) s += (double)x[c];
    s = block_sum(s);
    if (tid == 0) bc[0] = s / n;
    __syncthreads();
    const T xm = (T)bc[0];
    for (int c = tid; c < n; c += nt) x[c] -= xm;
}

// ---- dense coarsest-level solve --------------------------------------------
// M = A_c + s 1 1^T (SPD; on mean-free right sides M^{-1} f is the mean-free
// solution of A_c x = f, since the constants are an eigenvector of M with
// eigenvalue s n and the range of A_c is orthogonal to them).
// Row r = blockIdx.y, columns across x (the case along z).
template <class T, bool B>
__global__ void k_dense_assemble(Bat bt, Dims d, double ih2, const T* __restrict__ bx,
                                 const T* __restrict__ by, const T* __restrict__ bz, double s,
                                 T* __restrict__ M) {
    const BatBlk bb = bat_blk<B>(bt, blockIdx.z, gridDim.z);
    if (bb.off) return;
    bx = bat_at<B>(bt, bb.cs, bx);
    by = bat_at<B>(bt, bb.cs, by);
    bz = bat_at<B>(bt, bb.cs, bz);
    M = bat_at<B>(bt, bb.cs, M);
    const int n = d.nx * d.ny * d.nz;
    const int r = blockIdx.y;
    const int i = r % d.nx, j = (r / d.nx) % d.ny, k = r / (d.nx * d.ny);
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < n; col += gridDim.x * blockDim.x) {
        const long e = (long)r * n + col;
        double v = s;
        if (col == r) {
            v += ((double)bx[uid(d, i, j, k)] + bx[uid(d, i + 1, j, k)] + by[vid(d, i, j, k)] +
                  by[vid(d, i, j + 1, k)] + bz[wid(d, i, j, k)] +
                  bz[wid(d, i, j, wrapk(k + 1, d.nz))]) * ih2;
        } else {
            // the six neighbours (walls carry beta = 0; on a periodic axis of
            // length 2 both neighbours are the same cell and both faces count)
            if (i > 0 && col == r - 1) v -= (double)bx[uid(d, i, j, k)] * ih2;
            if (i < d.nx - 1 && col == r + 1) v -= (double)bx[uid(d, i + 1, j, k)] * ih2;
            if (j > 0 && col == r - d.nx) v -= (double)by[vid(d, i, j, k)] * ih2;
            if (j < d.ny - 1 && col == r + d.nx) v -= (double)by[vid(d, i, j + 1, k)] * ih2;
            if (col == cid(d, i, j, wrapk(k - 1, d.nz))) v -= (double)bz[wid(d, i, j, k)] * ih2;
            if (col == cid(d, i, j, wrapk(k + 1, d.nz)))
                v -= (double)bz[wid(d, i, j, wrapk(k + 1, d.nz))] * ih2;
        }
        M[e] = (T)v;
    }
}

// In-place Gauss-Jordan inversion of the SPD matrix (no pivoting needed):
// a pivot on index k maps M_kk -> 1/M_kk, row k -> row k / M_kk, column k ->
// -column k / M_kk and every other entry to M_ij - M_ik M_kj / M_kk; all n
// pivots leave M^-1.
// Blocked form of the same in-place inversion: pivoting on a block K of up
// to 32 indices at once (A = M_KK, B = M_KR, C = M_RK, D = M_RR) gives
//   M_KK <- A^-1,  M_KR <- A^-1 B,  M_RK <- -C A^-1,  M_RR <- D - C A^-1 B,
// which equals the 32 single-pivot steps in sequence. Two launches per block:
// the panel (A^-1 by 32 pivot steps in shared memory, padded with the
// identity, then -C A^-1 and A^-1 B) and the rank-32 update of the rest.
constexpr int GJB = 32;

template <class S, bool B>
__global__ void k_gj_panel(Bat bt, int n, int k, int bs, const S* __restrict__ M,
                           S* __restrict__ P, S* __restrict__ Cp, S* __restrict__ Bp) {
    const BatBlk bb = bat_blk<B>(bt, blockIdx.y, gridDim.y);
    if (bb.off) return;
    M = bat_at<B>(bt, bb.cs, M);
    P = bat_at<B>(bt, bb.cs, P);
    Cp = bat_at<B>(bt, bb.cs, Cp);
    Bp = bat_at<B>(bt, bb.cs, Bp);
    __shared__ S a[GJB][GJB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    a[ty][tx] = (ty < bs && tx < bs) ? M[(long)(k + ty) * n + k + tx] : S(ty == tx ? 1 : 0);
    for (int p = 0; p < GJB; ++p) {
        __syncthreads();
        const S r = S(1) / a[p][p];
        S v;
        if (ty == p && tx == p) v = r;
        else if (ty == p) v = a[p][tx] * r;
        else if (tx == p) v = -a[ty][p] * r;
        else v = a[ty][tx] - a[ty][p] * (a[p][tx] * r);
        __syncthreads();
        a[ty][tx] = v;
    }
    __syncthreads();
    if (blockIdx.x == 0) P[ty * GJB + tx] = a[ty][tx];
    const int i = blockIdx.x * GJB + ty;  // a row of -C A^-1
    if (i < n && tx < bs) {
        S v = S(0);
        if (i < k || i >= k + bs) {
            const S* row = M + (long)i * n + k;
            for (int t = 0; t < bs; ++t) v -= row[t] * a[t][tx];
        }
        Cp[(long)i * GJB + tx] = v;
    }
    const int j = blockIdx.x * GJB + tx;  // a column of A^-1 B
    if (j < n && ty < bs && (j < k || j >= k + bs)) {
        S v = S(0);
        for (int t = 0; t < bs; ++t) v += a[ty][t] * M[(long)(k + t) * n + j];
        Bp[(long)ty * n + j] = v;
    }
}

template <class S, bool B>
__global__ void k_gj_update(Bat bt, int n, int k, int bs, const S* __restrict__ M,
                            const S* __restrict__ P, const S* __restrict__ Cp,
                            const S* __restrict__ Bp, S* __restrict__ out) {
    const BatBlk bb = bat_blk<B>(bt, blockIdx.z, gridDim.z);
    if (bb.off) return;
    M = bat_at<B>(bt, bb.cs, M);
    P = bat_at<B>(bt, bb.cs, P);
    Cp = bat_at<B>(bt, bb.cs, Cp);
    Bp = bat_at<B>(bt, bb.cs, Bp);
    out = bat_at<B>(bt, bb.cs, out);
    __shared__ S cps[GJB][GJB + 1], mk[GJB][GJB + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * GJB + ty, j = blockIdx.x * GJB + tx;
    cps[ty][tx] = (i < n && tx < bs) ? Cp[(long)i * GJB + tx] : S(0);
    mk[ty][tx] = (ty < bs && j < n) ? M[(long)(k + ty) * n + j] : S(0);
    __syncthreads();
    if (i >= n || j >= n) return;
    const bool ki = i >= k && i < k + bs, kj = j >= k && j < k + bs;
    S v;
    if (ki && kj) v = P[(i - k) * GJB + (j - k)];
    else if (ki) v = Bp[(long)(i - k) * n + j];
    else if (kj) v = Cp[(long)i * GJB + (j - k)];
    else {
        v = M[(long)i * n + j];
        for (int u = 0; u < bs; ++u) v += cps[ty][u] * mk[u][tx];
    }
    out[(long)i * n + j] = v;
}

// x = Minv f: one warp per row (dense_row)
template <class T, bool B>
__global__ void k_dense_apply(Bat bt, int n, const T* __restrict__ Minv, const T* __restrict__ f,
                              T* __restrict__ x) {
    pdl_wait();
    const BatBlk bb = bat_blk<B>(bt, blockIdx.y, gridDim.y);
    if (bb.off) return;
    Minv = bat_at<B>(bt, bb.cs, Minv);
    f = bat_at<B>(bt, bb.cs, f);
    x = bat_at<B>(bt, bb.cs, x);
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double s = dense_row(Minv + (long)warp * n, [&](int j) { return f[j]; }, n, lane);
    if (lane == 0) x[warp] = (T)s;
}

template <class T>
__global__ void k_zero_t(int n, T* __restrict__ x) {
    pdl_wait();
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        x[c] = T(0);
}

// ---- inner FP32 Krylov kernels of the mixed-precision solve -----------------
// Per-thread partial sums are FP32 with Kahan compensation (on B300 an FP64
// add per element costs more than the memory traffic of these kernels); the
// block and grid sums of the partials are FP64.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// q = A32 p and the block partials of p.q (FP64 accumulation)
__global__ void k_apply_A_dot32(Dims d, float ih2, const float* __restrict__ bx,
                                const float* __restrict__ by, const float* __restrict__ bz,
                                const float* __restrict__ p, float* __restrict__ q,
                                double* __restrict__ part, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    Kahan ks;
    if (act)
        for (int k = k0; k < k1; ++k) {
            const int c = cid(d, i, j, k);
            const float v = stencil_t(d, bx, by, bz, p, i, j, k) * ih2;
            q[c] = v;
            ks.add(p[c] * v);
        }
    const double acc = block_sum(ks.value());
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear()] = acc;
}

// e += alpha p, r -= alpha q, partials of r.r
__global__ void k_cg_update32(int n, float* __restrict__ e, float* __restrict__ r,
                              const float* __restrict__ p, const float* __restrict__ q,
                              const double* __restrict__ scal, double* __restrict__ part) {
    const float al = (float)scal[S_ALPHA];
    Kahan ks;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        e[c] += al * p[c];
        const float rv = r[c] - al * q[c];
        r[c] = rv;
        ks.add(rv * rv);
    }
    const double acc = block_sum(ks.value());
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_dot2_32(int n, const float* __restrict__ z, const float* __restrict__ r,
                          const float* __restrict__ q, double* __restrict__ pa,
                          double* __restrict__ pb) {
    Kahan ka, kb;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const float zc = z[c];
        ka.add(zc * r[c]);
        kb.add(zc * q[c]);
    }
    const double a = block_sum(ka.value());
    const double b = block_sum(kb.value());
    if (threadIdx.x == 0) {
        pa[blockIdx.x] = a;
        pb[blockIdx.x] = b;
    }
}

__global__ void k_p_update32(int n, float* __restrict__ p, const float* __restrict__ z,
                             const double* __restrict__ scal) {
    const float be = (float)scal[S_BETA];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        p[c] = z[c] + be * p[c];
}

// the same with 16-byte loads and stores (n4 = n / 4, 16-byte aligned arrays)
template <bool B>
__global__ void k_p_update32x4(Bat t, int n4, float4* __restrict__ p,
                               const float4* __restrict__ z, const double* __restrict__ scal) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.y, gridDim.y);
    if (bb.off) return;
    p = bat_at<B>(t, bb.cs, p);
    z = bat_at<B>(t, bb.cs, z);
    scal = bat_at<B>(t, bb.cs, scal);
    const float be = (float)scal[S_BETA];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x) {
        const float4 zv = z[c];
        float4 pv = p[c];
        pv.x = zv.x + be * pv.x;
        pv.y = zv.y + be * pv.y;
        pv.z = zv.z + be * pv.z;
        pv.w = zv.w + be * pv.w;
        p[c] = pv;
    }
}

// k_cg_update32 with 16-byte loads and stores; each thread's (r, r) terms
// are summed four at a time, in order
template <bool B>
__global__ void k_cg_update32x4(Bat t, int n4, float4* __restrict__ e, float4* __restrict__ r,
                                const float4* __restrict__ p, const float4* __restrict__ q,
                                const double* __restrict__ scal, double* __restrict__ part) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.y, gridDim.y);
    if (bb.off) return;
    e = bat_at<B>(t, bb.cs, e);
    r = bat_at<B>(t, bb.cs, r);
    p = bat_at<B>(t, bb.cs, p);
    q = bat_at<B>(t, bb.cs, q);
    scal = bat_at<B>(t, bb.cs, scal);
    part = bat_at<B>(t, bb.cs, part);
    const float al = (float)scal[S_ALPHA];
    Kahan ks;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x) {
        const float4 pv = p[c], qv = q[c];
        float4 ev = e[c], rv = r[c];
        ev.x += al * pv.x;
        ev.y += al * pv.y;
        ev.z += al * pv.z;
        ev.w += al * pv.w;
        rv.x = rv.x - al * qv.x;
        rv.y = rv.y - al * qv.y;
        rv.z = rv.z - al * qv.z;
        rv.w = rv.w - al * qv.w;
        e[c] = ev;
        r[c] = rv;
        ks.add(rv.x * rv.x);
        ks.add(rv.y * rv.y);
        ks.add(rv.z * rv.z);
        ks.add(rv.w * rv.w);
    }
    const double acc = block_sum(ks.value());
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// 16-byte vector access is possible: n a multiple of 4, every array aligned
inline bool vec4_ok(int n, std::initializer_list<const void*> ptrs) {
    if (n % 4) return false;
    for (const void* q : ptrs)
        if (reinterpret_cast<uintptr_t>(q) % 16) return false;
    return true;
}

// x64 += e32 (the outer FP64 update of the defect correction)
__global__ void k_add_f32_to_f64(int n, const float* __restrict__ e, double* __restrict__ x) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        x[c] += (double)e[c];
}

__global__ void k_to_f32(int n, const double* __restrict__ a, float* __restrict__ b) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        b[c] = (float)a[c];
}

// FP16 copy of FP32 coefficients divided by a power of two (exact before the
// rounding to FP16)
__global__ void k_to_f16(int n, const float* __restrict__ a, __half* __restrict__ b, float inv_s) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        b[c] = __float2half_rn(a[c] * inv_s);
}

__global__ void k_to_f64(int n, const float* __restrict__ a, double* __restrict__ b) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        b[c] = (double)a[c];
}

// the same three with 16-byte accesses, four values per thread and pass
// (n4 = n / 4; arrays 16-byte aligned)
template <bool B>
__global__ void k_add_f32_to_f64x4(Bat t, int n4, const float4* __restrict__ e,
                                   double2* __restrict__ x) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.y, gridDim.y);
    if (bb.off) return;
    e = bat_at<B>(t, bb.cs, e);
    x = bat_at<B>(t, bb.cs, x);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x) {
        const float4 ev = e[c];
        double2 lo = x[2 * c], hi = x[2 * c + 1];
        lo.x += (double)ev.x;
        lo.y += (double)ev.y;
        hi.x += (double)ev.z;
        hi.y += (double)ev.w;
        x[2 * c] = lo;
        x[2 * c + 1] = hi;
    }
}

__global__ void k_to_f32x4(int n4, const double2* __restrict__ a, float4* __restrict__ b) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x) {
        const double2 lo = a[2 * c], hi = a[2 * c + 1];
        b[c] = make_float4((float)lo.x, (float)lo.y, (float)hi.x, (float)hi.y);
    }
}

__global__ void k_to_f64x4(int n4, const float4* __restrict__ a, double2* __restrict__ b) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x) {
        const float4 v = a[c];
        b[2 * c] = make_double2((double)v.x, (double)v.y);
        b[2 * c + 1] = make_double2((double)v.z, (double)v.w);
    }
}

inline int flat_blocks(int n) {
    int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 1184 ? 1184 : b);
}

template <class T>
struct LA {
    T *bx, *by, *bz, *x, *f;
};
template <class T>
LA<T> arrays(const Level& L);
template <>
LA<double> arrays<double>(const Level& L) {
    return {L.bx, L.by, L.bz, L.x, L.f};
}
template <>
LA<float> arrays<float>(const Level& L) {
    return {L.bxf, L.byf, L.bzf, L.xf, L.ff};
}

}  // namespace

// Levels narrower than FLAT_NX cells in x run their colour passes and the
// restriction from them a thread per (x-pair, y, z) or coarse cell in 1-D
// blocks (Level::pass_block, restrict_block threads), instead of 32 x 8
// tiles of which a 24- or 12-cell-wide plane fills a third or less.
constexpr int FLAT_NX = 64;

// one colour pass on a level with an even nx, a thread per x-pair; CT is
// the coefficients' storage type
template <class T, class CT>
void rbgs_pair(vof_ctx* c, const Level& L, T h2, const CT* bx, const CT* by, const CT* bz,
               const LA<T>& a, int color, int mode, const Level* C, int cls) {
    using K = void (*)(Bat, Dims, T, const CT*, const CT*, const CT*, const T*, T*, const T*, int,
                       int, Dims, const T*, T);
    const bool bat = c->bat_n > 1;
    const bool flat = L.d.nx < FLAT_NX;
    const K kern =
        flat ? (bat ? (mode == 1 ? k_rbgs_pair_t<T, 1, CT, true, true>
                                 : (mode == 2 ? k_rbgs_pair_t<T, 2, CT, true, true>
                                              : k_rbgs_pair_t<T, 0, CT, true, true>))
                    : (mode == 1 ? k_rbgs_pair_t<T, 1, CT, false, true>
                                 : (mode == 2 ? k_rbgs_pair_t<T, 2, CT, false, true>
                                              : k_rbgs_pair_t<T, 0, CT, false, true>)))
             : (bat ? (mode == 1 ? k_rbgs_pair_t<T, 1, CT, true>
                                 : (mode == 2 ? k_rbgs_pair_t<T, 2, CT, true>
                                              : k_rbgs_pair_t<T, 0, CT, true>))
                    : (mode == 1 ? k_rbgs_pair_t<T, 1, CT, false>
                                 : (mode == 2 ? k_rbgs_pair_t<T, 2, CT, false>
                                              : k_rbgs_pair_t<T, 0, CT, false>)));
    const Dims dc = C ? C->d : L.d;
    const T* xc = C ? arrays<T>(*C).x : nullptr;
    const T omega = (T)(c->sv.mg_omega > 0.0 ? c->sv.mg_omega : 1.0);
    int m = timer_begin(c, cls);
    if (flat) {
        const int nb = L.pass_block;
        dim3 grid((L.ncells / 2 + nb - 1) / nb);
        const Bat bt = bat_of(c, grid.y);
        launch_pdl(c, kern, grid, dim3(nb), bt, L.d, h2, bx, by, bz, (const T*)a.x, a.x,
                   a.f, color, 1, dc, xc, omega);
    } else {
        // a thread per x-pair halves the blocks of the level's cell geometry;
        // the z chunks are divided (by 4 unless timed or set otherwise) to
        // keep enough blocks in flight
        const int gx = (L.d.nx / 2 + TBX - 1) / TBX;
        const int kchunk = pass_kchunk_of(L);
        dim3 grid(gx, L.L.grid.y, (L.d.nz + kchunk - 1) / kchunk);
        const Bat bt = bat_of(c, grid.z);
        launch_pdl(c, kern, grid, L.L.block, bt, L.d, h2, bx, by, bz, (const T*)a.x, a.x, a.f,
                   color, kchunk, dc, xc, omega);
    }
    timer_end(c, cls, m);
}

template <class T>
void mg_rbgs(vof_ctx* c, const Level& L, int color, int mode, const Level* C) {
    const LA<T> a = arrays<T>(L);
    const int cls = L.idx == 0 ? T_SMOOTH0 : T_SMOOTH;
    if (L.d.nx % 2 != 0) {  // odd rows: separate zeroing / prolongation passes
        if (mode == 1) mg_zero<T>(c, L);
        if (mode == 2) mg_prolong<T>(c, *C, L);
        int m = timer_begin(c, cls);
        launch_pdl(c, k_rbgs_t<T>, L.L.grid, L.L.block, L.d, (T)(L.h * L.h), a.bx, a.by, a.bz,
                   a.x, a.f, color, L.L.kchunk);
        timer_end(c, cls, m);
        return;
    }
    if constexpr (sizeof(T) == sizeof(float)) {
        if (L.bxh) {
            // coefficients stored over s: the same update with h^2 / s
            rbgs_pair(c, L, (T)(L.h * L.h) / L.hscale, L.bxh, L.byh, L.bzh, a, color, mode, C,
                      cls);
            return;
        }
    }
    rbgs_pair(c, L, (T)(L.h * L.h), a.bx, a.by, a.bz, a, color, mode, C, cls);
}

template <class T>
void mg_restrict(vof_ctx* c, const Level& F, const Level& C) {
    const LA<T> a = arrays<T>(F), b = arrays<T>(C);
    const int cls = F.idx == 0 ? T_RESTRICT0 : T_RESTRICT;
    int m = timer_begin(c, cls);
    if (c->sv.mg_interp == VOF_MG_TRILINEAR) {
        T* r = (T*)F.rs;
        VOF_LAUNCH(c, k_mg_residual_t<T>, F.L.grid, F.L.block, F.d, (T)(1.0 / (F.h * F.h)), a.bx,
                   a.by, a.bz, a.x, a.f, r, F.L.kchunk);
        VOF_LAUNCH(c, k_restrict_fw_t<T>, C.L.grid, C.L.block, F.d, (const T*)r, C.d, b.f,
                   C.L.kchunk);
    } else {
        dim3 g = C.L.grid;
        if (sizeof(T) == sizeof(float) && F.bxh) {
            const Bat bt = bat_of(c, g.z);
            launch_pdl(c, bt.zb ? k_restrict_pair_f<__half, true> : k_restrict_pair_f<__half, false>,
                       g, C.L.block, bt, F.d,
                       (float)(1.0 / (F.h * F.h)) * F.hscale, (const __half*)F.bxh, (const __half*)F.byh,
                       (const __half*)F.bzh, (const float*)a.x, (const float*)a.f, C.d,
                       (float*)b.f, C.L.kchunk);
        } else if (sizeof(T) == sizeof(float) && F.d.nx % 2 == 0 && F.d.nx < FLAT_NX) {
            const int nb = F.restrict_block;
            dim3 gf((C.ncells + nb - 1) / nb);
            const Bat bt = bat_of(c, gf.y);
            launch_pdl(c, bt.zb ? k_restrict_pair_f<float, true, true>
                                : k_restrict_pair_f<float, false, true>,
                       gf, dim3(nb), bt, F.d, (float)(1.0 / (F.h * F.h)),
                       (const float*)a.bx, (const float*)a.by, (const float*)a.bz,
                       (const float*)a.x, (const float*)a.f, C.d, (float*)b.f, 1);
        } else if (sizeof(T) == sizeof(float) && F.d.nx % 2 == 0) {
            const Bat bt = bat_of(c, g.z);
            launch_pdl(c, bt.zb ? k_restrict_pair_f<float, true> : k_restrict_pair_f<float, false>,
                       g, C.L.block, bt, F.d,
                       (float)(1.0 / (F.h * F.h)), (const float*)a.bx, (const float*)a.by,
                       (const float*)a.bz, (const float*)a.x, (const float*)a.f, C.d, (float*)b.f,
                       C.L.kchunk);
        }
        else
            launch_pdl(c, k_restrict_t<T>, C.L.grid, C.L.block, F.d, (T)(1.0 / (F.h * F.h)),
                       a.bx, a.by, a.bz, a.x, a.f, C.d, b.f, C.L.kchunk);
    }
    timer_end(c, cls, m);
}

template <class T>
void mg_prolong(vof_ctx* c, const Level& C, const Level& F) {
    const LA<T> a = arrays<T>(C), b = arrays<T>(F);
    const int cls = F.idx == 0 ? T_PROLONG0 : T_PROLONG;
    int m = timer_begin(c, cls);
    const T omega = (T)(c->sv.mg_omega > 0.0 ? c->sv.mg_omega : 1.0);
    if (c->sv.mg_interp == VOF_MG_TRILINEAR)
        VOF_LAUNCH(c, k_prolong_tri_t<T>, F.L.grid, F.L.block, C.d, a.x, F.d, b.x, omega,
                   F.L.kchunk);
    else if (sizeof(T) == sizeof(float) && F.d.nx % 2 == 0) {
        const int kchunk = std::max(1, (F.L.kchunk + 1) / 2);  // half the blocks across
        dim3 g((F.d.nx / 2 + TBX - 1) / TBX, F.L.grid.y, (F.d.nz + kchunk - 1) / kchunk);
        const Bat bt = bat_of(c, g.z);
        launch_pdl(c, bt.zb ? k_prolong_pair_f<true> : k_prolong_pair_f<false>, g, F.L.block, bt,
                   C.d, (const float*)a.x, F.d,
                   (float*)b.x, (float)omega, kchunk);
    }
    else
        launch_pdl(c, k_prolong_t<T>, F.L.grid, F.L.block, C.d, a.x, F.d, b.x, omega, F.L.kchunk);
    timer_end(c, cls, m);
}

template <class T>
void mg_coarsen_beta(vof_ctx* c, const Level& F, const Level& C) {
    const LA<T> a = arrays<T>(F), b = arrays<T>(C);
    VOF_LAUNCH(c, k_coarsen_beta_t<T>, C.L.grid, C.L.block, F.d, a.bx, a.by, a.bz, C.d, b.bx, b.by,
               b.bz, C.L.kchunk);
}

template <class T>
void mg_coarsen_density(vof_ctx* c, const T* rf, const Level& F, const Level& C) {
    const LA<T> b = arrays<T>(C);
    VOF_LAUNCH(c, k_avg8_t<T>, C.L.grid, C.L.block, F.d, rf, C.d, (T*)C.rho, C.L.kchunk);
    VOF_LAUNCH(c, k_beta_from_rho_t<T>, C.L.grid, C.L.block, C.d, (const T*)C.rho, b.bx, b.by,
               b.bz, C.L.kchunk);
}
template void mg_coarsen_density<double>(vof_ctx*, const double*, const Level&, const Level&);
template void mg_coarsen_density<float>(vof_ctx*, const float*, const Level&, const Level&);

// FP64 finest-level coefficients averaged straight into the FP32 level 1
// (the mixed V-cycle's finest level keeps no FP32 face arrays)
void mg_coarsen_beta_from64(vof_ctx* c, const Level& F, const Level& C) {
    void (*const kern)(Dims, const double*, const double*, const double*, Dims, float*, float*,
                       float*, int) = k_coarsen_beta_t<float, double>;
    VOF_LAUNCH(c, kern, C.L.grid, C.L.block, F.d, F.bx, F.by, F.bz, C.d, C.bxf, C.byf, C.bzf,
               C.L.kchunk);
}

// Factor the coarsest level once per solve: explicit inverse of A_c + s 11^T
// by Gauss-Jordan in the V-cycle's precision (FP64 path: FP64; mixed path:
// FP32, an inverse accurate to about cond * eps_32, ample for a
// preconditioner whose outer iteration is FP64).
template <class T>
void mg_dense_setup(vof_ctx* c, const Level& L) {
    const LA<T> a = arrays<T>(L);
    const int n = L.ncells;
    const double ih2 = 1.0 / (L.h * L.h);
    // s n: the liquid-coefficient scale of the diagonal, so the constants'
    // eigenvalue of the shifted matrix sits among the operator's own
    const double s = c->dense_shift * ih2 / n;
    int m = timer_begin(c, T_COARSE);
    T* A = (T*)c->dense_a;
    T* B = (T*)c->dense_b;
    const bool bat = c->bat_n > 1;
    dim3 ga((n + 255) / 256, n);
    const Bat bta = bat_of(c, ga.z);
    auto kas = bat ? k_dense_assemble<T, true> : k_dense_assemble<T, false>;
    VOF_LAUNCH(c, kas, ga, 256, bta, L.d, ih2, a.bx, a.by, a.bz, s, A);
    T* Pw = (T*)c->dense_w;
    T* Cp = Pw + GJB * GJB;
    T* Bp = Cp + (size_t)GJB * n;
    const int nt = (n + GJB - 1) / GJB;
    for (int k = 0; k < n; k += GJB) {
        const int bs = std::min(GJB, n - k);
        dim3 gp(nt), gu(nt, nt);
        const Bat btp = bat_of(c, gp.y), btu = bat_of(c, gu.z);
        auto kp = bat ? k_gj_panel<T, true> : k_gj_panel<T, false>;
        auto ku = bat ? k_gj_update<T, true> : k_gj_update<T, false>;
        VOF_LAUNCH(c, kp, gp, dim3(GJB, GJB), btp, n, k, bs, (const T*)A, Pw, Cp, Bp);
        VOF_LAUNCH(c, ku, gu, dim3(GJB, GJB), btu, n, k, bs, (const T*)A, (const T*)Pw,
                   (const T*)Cp, (const T*)Bp, B);
        std::swap(A, B);
    }
    if (sizeof(T) == 4) c->dense_inv_f = (float*)A;
    else c->dense_inv = (double*)A;
    timer_end(c, T_COARSE, m);
}

template <class T>
void mg_coarse(vof_ctx* c, const Level& L) {
    const LA<T> a = arrays<T>(L);
    int m = timer_begin(c, T_COARSE);
    if (c->dense_n > 0) {
        const int n = L.ncells;
        const T* Minv = sizeof(T) == 4 ? (const T*)c->dense_inv_f : (const T*)c->dense_inv;
        dim3 g((n * 32 + 255) / 256);
        const Bat bt = bat_of(c, g.y);
        launch_pdl(c, bt.zb ? k_dense_apply<T, true> : k_dense_apply<T, false>, g, dim3(256), bt, n,
                   Minv, a.f, a.x);
        timer_end(c, T_COARSE, m);
        return;
    }
    // default targets: FP64 tight, FP32 what single precision can hold
    const double tol = c->sv.coarse_tol > 0.0 ? c->sv.coarse_tol : (sizeof(T) == 8 ? 1e-8 : 1e-5);
    const int maxit = c->sv.coarse_iters > 0 ? c->sv.coarse_iters : 400;
    VOF_LAUNCH(c, k_coarse_cg_t<T>, 1, 1024, L.d, (T)(1.0 / (L.h * L.h)), a.bx, a.by, a.bz, a.f,
               a.x, (T*)c->coarse_scratch, maxit, tol);
    timer_end(c, T_COARSE, m);
}

template <class T>
void mg_zero(vof_ctx* c, const Level& L) {
    const LA<T> a = arrays<T>(L);
    launch_pdl(c, k_zero_t<T>, dim3(flat_blocks(L.ncells)), dim3(256), L.ncells, a.x);
}

void k32_apply_A_dot(vof_ctx* c, const float* p, float* q, int slot) {
    const Level& L = c->lv[0];
    int m = timer_begin(c, T_RESIDUAL);
    VOF_LAUNCH(c, k_apply_A_dot32, L.L.grid, L.L.block, L.d, (float)(1.0 / (L.h * L.h)), L.bxf,
               L.byf, L.bzf, p, q, c->part + (size_t)slot * MAX_PARTIALS, L.L.kchunk);
    timer_end(c, T_RESIDUAL, m);
    finalize_pq_alpha(c, L.L.nblocks);
}

int k32_cg_update(vof_ctx* c, int n, float* e, float* r, const float* p, const float* q, int slot,
                  bool finalize) {
    const bool v4 = vec4_ok(n, {e, r, p, q});
    const int nb = flat_blocks(v4 ? n / 4 : n);
    int m = timer_begin(c, T_KRYLOV);
    if (v4) {
        dim3 g(nb);
        const Bat b = bat_of(c, g.y);
        auto kern = b.zb ? k_cg_update32x4<true> : k_cg_update32x4<false>;
        VOF_LAUNCH(c, kern, g, 256, b, n / 4, (float4*)e, (float4*)r, (const float4*)p,
                   (const float4*)q, c->scal, c->part + (size_t)slot * MAX_PARTIALS);
    } else
        VOF_LAUNCH(c, k_cg_update32, nb, 256, n, e, r, p, q, c->scal,
                   c->part + (size_t)slot * MAX_PARTIALS);
    timer_end(c, T_KRYLOV, m);
    if (finalize) finalize_sum(c, slot, nb, slot, 1.0);
    return nb;
}

void k32_dot2(vof_ctx* c, int n, const float* z, const float* r, const float* q) {
    const int nb = flat_blocks(n);
    int m = timer_begin(c, T_KRYLOV);
    VOF_LAUNCH(c, k_dot2_32, nb, 256, n, z, r, q, c->part + (size_t)S_RZ * MAX_PARTIALS,
               c->part + (size_t)S_ZQ * MAX_PARTIALS);
    timer_end(c, T_KRYLOV, m);
    finalize_dots_beta(c, nb);
}

void k32_p_update(vof_ctx* c, int n, float* p, const float* z) {
    int m = timer_begin(c, T_KRYLOV);
    if (vec4_ok(n, {p, z})) {
        dim3 g(flat_blocks(n / 4));
        const Bat b = bat_of(c, g.y);
        auto kern = b.zb ? k_p_update32x4<true> : k_p_update32x4<false>;
        VOF_LAUNCH(c, kern, g, 256, b, n / 4, (float4*)p, (const float4*)z, c->scal);
    } else
        VOF_LAUNCH(c, k_p_update32, flat_blocks(n), 256, n, p, z, c->scal);
    timer_end(c, T_KRYLOV, m);
}

void k32_add_to_f64(vof_ctx* c, int n, const float* e, double* x) {
    int m = timer_begin(c, T_KRYLOV);
    if (vec4_ok(n, {e, x})) {
        dim3 g(flat_blocks(n / 4));
        const Bat b = bat_of(c, g.y);
        auto kern = b.zb ? k_add_f32_to_f64x4<true> : k_add_f32_to_f64x4<false>;
        VOF_LAUNCH(c, kern, g, 256, b, n / 4, (const float4*)e, (double2*)x);
    } else
        VOF_LAUNCH(c, k_add_f32_to_f64, flat_blocks(n), 256, n, e, x);
    timer_end(c, T_KRYLOV, m);
}

void mg_to_f32(vof_ctx* c, const double* a, float* b, int n) {
    if (vec4_ok(n, {a, b}))
        VOF_LAUNCH(c, k_to_f32x4, flat_blocks(n / 4), 256, n / 4, (const double2*)a, (float4*)b);
    else
        VOF_LAUNCH(c, k_to_f32, flat_blocks(n), 256, n, a, b);
}

void mg_half_coefficients(vof_ctx* c) {
    for (const Level& L : c->lv) {
        if (!L.bxh) continue;
        const int nu = (L.d.nx + 1) * L.d.ny * L.d.nz, nv = L.d.nx * (L.d.ny + 1) * L.d.nz;
        const float inv_s = 1.f / L.hscale;
        VOF_LAUNCH(c, k_to_f16, flat_blocks(nu), 256, nu, L.bxf, L.bxh, inv_s);
        VOF_LAUNCH(c, k_to_f16, flat_blocks(nv), 256, nv, L.byf, L.byh, inv_s);
        VOF_LAUNCH(c, k_to_f16, flat_blocks(L.ncells), 256, L.ncells, L.bzf, L.bzh, inv_s);
    }
}

void mg_to_f64(vof_ctx* c, const float* a, double* b, int n) {
    if (vec4_ok(n, {a, b}))
        VOF_LAUNCH(c, k_to_f64x4, flat_blocks(n / 4), 256, n / 4, (const float4*)a, (double2*)b);
    else
        VOF_LAUNCH(c, k_to_f64, flat_blocks(n), 256, n, a, b);
}

template void mg_rbgs<double>(vof_ctx*, const Level&, int, int, const Level*);
template void mg_rbgs<float>(vof_ctx*, const Level&, int, int, const Level*);
template void mg_restrict<double>(vof_ctx*, const Level&, const Level&);
template void mg_restrict<float>(vof_ctx*, const Level&, const Level&);
template void mg_prolong<double>(vof_ctx*, const Level&, const Level&);
template void mg_prolong<float>(vof_ctx*, const Level&, const Level&);
template void mg_coarsen_beta<double>(vof_ctx*, const Level&, const Level&);
template void mg_coarsen_beta<float>(vof_ctx*, const Level&, const Level&);
template void mg_coarse<double>(vof_ctx*, const Level&);
template void mg_coarse<float>(vof_ctx*, const Level&);
template void mg_zero<double>(vof_ctx*, const Level&);
template void mg_dense_setup<double>(vof_ctx*, const Level&);
template void mg_dense_setup<float>(vof_ctx*, const Level&);
template void mg_zero<float>(vof_ctx*, const Level&);

// ---------------------------------------------------------------------------
// Launch shapes of the coarse levels' colour passes, chosen by timing. A
// colour pass and the 1-D restriction are pointwise: each thread writes its
// own cells from loads, with the same rounded operations whatever the
// mapping, so the shape changes the time and never a bit. The choices are
// cached for the process per device, level dimensions, number of cases and
// storage types, so contexts of one shape (a server's requests, an
// ensemble's cases) time a level once.
namespace {

struct ShapeKey {
    int dev, nx, ny, nz, nb, tsize, half, kind;  // kind 0: colour passes, 1: restriction
    bool operator==(const ShapeKey& o) const {
        return dev == o.dev && nx == o.nx && ny == o.ny && nz == o.nz && nb == o.nb &&
               tsize == o.tsize && half == o.half && kind == o.kind;
    }
};
std::mutex g_shape_mu;
std::vector<std::pair<ShapeKey, int>> g_shapes;

bool cached_shape(const ShapeKey& k, int* v) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    for (const auto& e : g_shapes)
        if (e.first == k) {
            *v = e.second;
            return true;
        }
    return false;
}

void cache_shape(const ShapeKey& k, int v) {
    std::lock_guard<std::mutex> lk(g_shape_mu);
    for (auto& e : g_shapes)
        if (e.first == k) {
            e.second = v;
            return;
        }
    g_shapes.push_back({k, v});
}

// finite, normal values in a level's arrays for the timed passes: every
// coefficient byte 0x3C (1.06 in FP16, 0.0115 in FP32, 1.6e-18 in FP64),
// x and f zero (so the passes keep x at zero)
template <class T>
void fill_for_timing(vof_ctx* c, const Level& L) {
    const LA<T> a = arrays<T>(L);
    const size_t nu = (size_t)(L.d.nx + 1) * L.d.ny * L.d.nz;
    const size_t nv = (size_t)L.d.nx * (L.d.ny + 1) * L.d.nz;
    const size_t n = L.ncells;
    cudaMemsetAsync(a.bx, 0x3C, sizeof(T) * nu, c->st);
    cudaMemsetAsync(a.by, 0x3C, sizeof(T) * nv, c->st);
    cudaMemsetAsync(a.bz, 0x3C, sizeof(T) * n, c->st);
    cudaMemsetAsync(a.x, 0, sizeof(T) * n, c->st);
    cudaMemsetAsync(a.f, 0, sizeof(T) * n, c->st);
    if (sizeof(T) == sizeof(float) && L.bxh) {
        cudaMemsetAsync(L.bxh, 0x3C, sizeof(__half) * nu, c->st);
        cudaMemsetAsync(L.byh, 0x3C, sizeof(__half) * nv, c->st);
        cudaMemsetAsync(L.bzh, 0x3C, sizeof(__half) * n, c->st);
    }
}

// milliseconds of `reps` runs of op after one untimed run; negative on a
// CUDA error
template <class F>
float time_op(vof_ctx* c, cudaEvent_t e0, cudaEvent_t e1, int reps, F op) {
    op();
    cudaEventRecord(e0, c->st);
    for (int r = 0; r < reps; ++r) op();
    cudaEventRecord(e1, c->st);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        return -1.f;
    return ms;
}

// the fastest of the candidate values set by `set` (three interleaved
// rounds, the minimum of each candidate's times), or the built-in value
// `dflt` unless a candidate beats it by 5%; dflt on any error
template <class S, class F>
int pick(vof_ctx* c, cudaEvent_t e0, cudaEvent_t e1, int reps, const int* cand, int ncand,
         int dflt, S set, F op, bool* err) {
    float best[8];
    for (int i = 0; i < ncand; ++i) best[i] = 1e30f;
    for (int round = 0; round < 3; ++round)
        for (int i = 0; i < ncand; ++i) {
            set(cand[i]);
            const float ms = time_op(c, e0, e1, reps, op);
            if (ms < 0.f) {
                *err = true;
                set(dflt);
                return dflt;
            }
            best[i] = std::min(best[i], ms);
        }
    int bi = -1, di = -1;
    for (int i = 0; i < ncand; ++i) {
        if (cand[i] == dflt) di = i;
        if (bi < 0 || best[i] < best[bi]) bi = i;
    }
    const int v = (di < 0 || best[bi] < 0.95f * best[di]) ? cand[bi] : dflt;
    set(v);
    return v;
}

template <class T>
vof_status tune_levels(vof_ctx* c, int nb) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VOF_ERR_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return VOF_ERR_CUDA;
    }
    static const int kFlat[4] = {64, 128, 256, 512};
    static const int kRestrict[3] = {64, 128, 256};
    bool err = false;
    const int nl = (int)c->lv.size();
    for (int l = 1; l + 1 < nl && !err; ++l) {
        if (c->tail_level > 0 && l >= c->tail_level) break;  // visited by one tail launch
        Level& L = c->lv[l];
        if (L.d.nx % 2 != 0) continue;
        const bool flat = L.d.nx < FLAT_NX;
        const bool half = sizeof(T) == sizeof(float) && L.bxh;
        // about 2M cell updates per timing, at least 3 and at most 20 pass pairs
        const long long cells = std::max(1LL, (long long)L.ncells * nb);
        const int reps = (int)std::min(20LL, std::max(3LL, (2LL << 20) / cells));
        ShapeKey k{dev, L.d.nx, L.d.ny, L.d.nz, nb, (int)sizeof(T), half ? 1 : 0, 0};
        int v = 0;
        if (cached_shape(k, &v)) {
            (flat ? L.pass_block : L.pass_kchunk) = v;
        } else {
            auto pair = [&] {
                mg_rbgs<T>(c, L, 0, 0);
                mg_rbgs<T>(c, L, 1, 0);
            };
            if (flat) {
                v = pick(c, e0, e1, reps, kFlat, 4, 256, [&](int b) { L.pass_block = b; }, pair, &err);
            } else {
                // the level's z chunk divided by 1, 2, 4 (built in) or 8
                int kz[4];
                for (int i = 0; i < 4; ++i) {
                    kz[i] = std::max(1, (L.L.kchunk + (1 << i) - 1) >> i);
                    // grid z extent (chunks x cases) within the launch limit
                    if ((long long)((L.d.nz + kz[i] - 1) / kz[i]) * nb > 65535) kz[i] = L.L.kchunk;
                }
                v = pick(c, e0, e1, reps, kz, 4, kz[2], [&](int q) { L.pass_kchunk = q; }, pair,
                         &err);
            }
            if (!err) cache_shape(k, v);
        }
        L.tuned = !err;
        // the 1-D restriction from this level (FP32 coefficients, constant prolongation)
        if (sizeof(T) == sizeof(float) && flat && !L.bxh && c->sv.mg_interp != VOF_MG_TRILINEAR &&
            !err) {
            k.kind = 1;
            if (cached_shape(k, &v)) {
                L.restrict_block = v;
            } else {
                const Level& C = c->lv[l + 1];
                v = pick(c, e0, e1, 2 * reps, kRestrict, 3, 256,
                         [&](int b) { L.restrict_block = b; },
                         [&] { mg_restrict<T>(c, L, C); }, &err);
                if (!err) cache_shape(k, v);
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err ? VOF_ERR_CUDA : VOF_OK;
}

}  // namespace

vof_status mg_tune_shapes(vof_ctx* c, int nb, long long stride, int* act_d) {
    if (c->sv.mg_tune == VOF_TUNE_OFF || c->lv.size() < 3) return VOF_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->st, &cs) != cudaSuccess) return VOF_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return VOF_OK;  // no timing inside a capture
    const bool mixed = c->sv.precision == VOF_PREC_MIXED_FP32;
    if (nb <= 1) {
        // every case's arrays are filled by its own context before a batched
        // launch through case 0's reads them
        for (size_t l = 1; l < c->lv.size(); ++l) {
            if (mixed) fill_for_timing<float>(c, c->lv[l]);
            else fill_for_timing<double>(c, c->lv[l]);
        }
    } else {
        std::vector<int> on(nb, 1);
        if (cudaMemcpyAsync(act_d, on.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess)
            return VOF_ERR_CUDA;
        c->bat_n = nb;
        c->bat_stride = stride;
        c->bat_act = act_d;
    }
    const vof_status st = mixed ? tune_levels<float>(c, nb) : tune_levels<double>(c, nb);
    c->bat_n = 1;
    c->bat_stride = 0;
    c->bat_act = nullptr;
    return st;
}

vof_status mg_shape_of(const vof_ctx* c, int level, int shape[4]) {
    if (!c || !shape || level < 1 || level + 1 >= (int)c->lv.size()) return VOF_ERR_ARG;
    const Level& L = c->lv[level];
    if (L.d.nx % 2 != 0) return VOF_ERR_ARG;
    const bool flat = L.d.nx < FLAT_NX;
    const bool mixed = c->sv.precision == VOF_PREC_MIXED_FP32;
    shape[0] = flat ? 0 : pass_kchunk_of(L);
    shape[1] = flat ? L.pass_block : 0;
    shape[2] = (mixed && flat && !L.bxh && c->sv.mg_interp != VOF_MG_TRILINEAR) ? L.restrict_block : 0;
    shape[3] = L.tuned ? 1 : 0;
    return VOF_OK;
}

vof_status mg_set_shape(vof_ctx* c, int level, const int shape[3]) {
    int cur[4];
    const vof_status st = mg_shape_of(c, level, cur);
    if (st != VOF_OK) return st;
    Level& L = c->lv[level];
    auto block_ok = [](int b) { return b >= 32 && b <= 1024 && b % 32 == 0; };
    // a value must be given exactly where the level uses one
    if ((cur[0] == 0) != (shape[0] == 0) || (cur[1] == 0) != (shape[1] == 0) ||
        (cur[2] == 0) != (shape[2] == 0))
        return VOF_ERR_ARG;
    if (shape[0] && (shape[0] < 1 || shape[0] > L.d.nz || (L.d.nz + shape[0] - 1) / shape[0] > 65535))
        return VOF_ERR_ARG;
    if ((shape[1] && !block_ok(shape[1])) || (shape[2] && !block_ok(shape[2]))) return VOF_ERR_ARG;
    if (shape[0]) L.pass_kchunk = shape[0];
    if (shape[1]) L.pass_block = shape[1];
    if (shape[2]) L.restrict_block = shape[2];
    L.tuned = false;
    return VOF_OK;
}

int pass_kchunk_of(const Level& L) {
    return L.pass_kchunk > 0 ? L.pass_kchunk : std::max(1, (L.L.kchunk + 3) / 4);
}
