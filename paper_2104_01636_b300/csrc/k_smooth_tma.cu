// Finest level of the mixed-precision V-cycle (pressure equation, Eq. 7):
// the face coefficients are formed on the fly from one density per cell,
//   beta_f = 1 / (0.5 (rho_L + rho_R)) = 2 / (rho_L + rho_R),
// the same face rule as the FP64 coefficients (rho the linear mix of the two
// phases by the volume fraction), so a kernel reads one value per cell
// instead of three face arrays.
//
//  * k_sweep_rho: one whole red-black Gauss-Seidel sweep per launch (first
//    colour from the other colour's old values, then the other colour from
//    the new ones). A block owns a 32 x 32 (x, y) tile and marches over a
//    chunk of z planes; TMA (cp.async.bulk.tensor) stages the planes of x
//    (FP32) and of the density (FP16), halo included, in shared memory. The
//    first colour is computed on the tile and on its one-cell ring (the ring
//    redundantly with the neighbouring tiles), so a block never reads
//    another block's result; x is read from one buffer and written to
//    another, and the result does not depend on the order in which blocks
//    run.
//  * k_restrict_rho: residual f - A x averaged over the eight children.
//    With the sweep it forms the V-cycle's finest-level operator from the
//    FP16 density (a preconditioner: the 11-bit density changes no
//    convergence test), so the V-cycle stays symmetric.
//  * k_apply_A_dot_rho32_pair: q = A p with the partials of p.q, from the FP32
//    density: the inner CG's operator, which the FP64 defect correction
//    must see to within FP32 rounding.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "vof_internal.cuh"

namespace {

constexpr int STX = 32, STY = 32;            // tile of a sweep block
constexpr int SBX = STX + 8, SBY = STY + 4;   // x box (FP32): x from i0-4 (16-byte aligned), y from j0-2
constexpr int HBX = STX + 16;                 // density box (FP16): x from i0-8 (16-byte aligned)
constexpr int RNX = STX + 2, RNY = STY + 2;   // the tile and its ring
constexpr int NCX = RNX / 2;                  // first-colour cells per ring-region row (stored compactly)
constexpr int NPL = NCX * RNY;                // floats per first-colour plane
constexpr int NSLOT = 4;                      // staged planes: 3 in use, 1 in flight
constexpr int XPLANE = SBX * SBY;             // floats per staged x plane
constexpr int HPLANE = HBX * SBY;             // halves per staged density plane
constexpr int WAIT_LIMIT = 1 << 20;           // bounded waits on the TMA barriers
constexpr int SWEEP_BLOCKS_PER_SM = 4;        // resident sweep blocks per SM (registers <= 64)
constexpr size_t SWEEP_SMEM = (size_t)NSLOT * XPLANE * sizeof(float) +
                              (size_t)NSLOT * HPLANE * sizeof(__half) +
                              (size_t)3 * NPL * sizeof(float) + NSLOT * sizeof(uint64_t) + 128;
static_assert(sizeof(CUtensorMap) == 128, "tensor map storage in the context is 128 bytes");
static_assert((SBX * sizeof(float)) % 16 == 0 && (HBX * sizeof(__half)) % 16 == 0,
              "TMA box rows must be a multiple of 16 bytes");
static_assert(SWEEP_SMEM + 1024 <= 228 * 1024 / SWEEP_BLOCKS_PER_SM,
              "shared memory of SWEEP_BLOCKS_PER_SM resident sweep blocks");
static_assert((XPLANE * sizeof(float)) % 128 == 0 && (HPLANE * sizeof(__half)) % 128 == 0,
              "staged planes keep 128-byte alignment");

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// the face coefficient 2 / (rho_L + rho_R); the sweep uses its exact half
__device__ __forceinline__ float beta_rho(float rc, float rn) { return 2.f * rcp_approx(rc + rn); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// a box of plane z of case w (the fourth axis: the cases of a batched
// launch, 0 for a single case)
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
        : "memory");
}

struct SweepArgs {
    int nx, ny, nz;
    float h2half;  // h^2 / 2: the sweep works with half coefficients 1 / (rho_L + rho_R)
    int c0;        // colour updated first: cells with (i + j + k) % 2 == c0
    int kchunk;
    const float* f;
    float* xout;
    double* err;  // set to 1 when a wait on a TMA barrier gives up
    // DOT sweeps: block partials of (x_new, f) and (x_new, q) into pa, pb
    const float* q;
    double *pa, *pb;
    Bat bt;  // the batch (Bat{} for a single case); the TMA maps carry the cases as a fourth axis
};

// 1 / (rho_L + rho_R), half the face coefficient: every finest-level kernel
// forms its coefficients through this one expression
__device__ __forceinline__ float half_beta(float rc, float rn) { return rcp_approx(rc + rn); }

__device__ __forceinline__ float2 half_beta2(float2 rc, float2 rn) {
    const float2 s = __fadd2_rn(rc, rn);
    return make_float2(rcp_approx(s.x), rcp_approx(s.y));
}

__device__ __forceinline__ float hval(const __half* h, int o) { return __half2float(h[o]); }

// Each thread owns the x-pair (ib, ib+1) in rows jA = j0+ty and jB = jA+16.
// On every plane one member of the pair has the first colour and the other
// the second, at the same x in both rows, so the two rows are updated with
// packed FP32x2 arithmetic. The z-face coefficients computed for the first
// colour are kept in registers and reused by the second colour, and the
// right side of the next plane is loaded into registers one plane ahead.
// DOT: as the pair is written, its products with f and with q are summed
// (the preconditioner's last sweep forms the Krylov dots (z, r), (z, q)
// from the z it writes, r being its right side).
template <bool ZERO, bool DOT, bool B>
__global__ void __launch_bounds__(256, SWEEP_BLOCKS_PER_SM)
    k_sweep_rho(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_rho,
                SweepArgs a0) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    float* sX = reinterpret_cast<float*>(smem_raw + (((raw + 127u) & ~127u) - raw));
    __half* sH = reinterpret_cast<__half*>(sX + NSLOT * XPLANE);
    float* sN = reinterpret_cast<float*>(sH + NSLOT * HPLANE);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sN + 3 * NPL);

    const BatBlk bb = bat_blk<B>(a0.bt, blockIdx.z, gridDim.z);
    if (bb.off) return;
    SweepArgs a = a0;
    a.f = bat_at<B>(a0.bt, bb.cs, a0.f);
    a.xout = bat_at<B>(a0.bt, bb.cs, a0.xout);
    a.err = bat_at<B>(a0.bt, bb.cs, a0.err);
    a.q = bat_at<B>(a0.bt, bb.cs, a0.q);
    a.pa = bat_at<B>(a0.bt, bb.cs, a0.pa);
    a.pb = bat_at<B>(a0.bt, bb.cs, a0.pb);
    const int blin = block_linear_z(bb);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 16 * ty;
    const int i0 = blockIdx.x * STX, j0 = blockIdx.y * STY;
    const int k0 = bb.b * a.kchunk;
    const int k1 = min(k0 + a.kchunk, a.nz);
    if (k0 >= k1) {  // whole block
        if (DOT && threadIdx.x == 0 && threadIdx.y == 0) a.pa[blin] = a.pb[blin] = 0.0;
        return;
    }
    const int pbase = k0 - 2;  // first staged plane (unwrapped index)
    constexpr uint32_t bytes = (ZERO ? 0u : (uint32_t)(XPLANE * sizeof(float))) +
                               (uint32_t)(HPLANE * sizeof(__half));

    if (tid == 0) {
        for (int s = 0; s < NSLOT; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    int issued = pbase - 1;  // last plane issued (thread 0)
    auto issue = [&](int p) {
        const int s = (p - pbase) % NSLOT;
        const int z = wrapk(p, a.nz);
        mbar_expect_tx(&bar[s], bytes);
        if (!ZERO) tma_load_4d(sX + s * XPLANE, &tm_x, &bar[s], i0 - 4, j0 - 2, z, bb.cs);
        tma_load_4d(sH + s * HPLANE, &tm_rho, &bar[s], i0 - 8, j0 - 2, z, bb.cs);
        issued = p;
    };
    if (tid == 0)
        for (int p = pbase; p <= pbase + NSLOT - 1; ++p) issue(p);

    bool bad = false;
    auto wait_slot = [&](int s, uint32_t par) {
        for (int it = 0; !bad && !mbar_try_wait(&bar[s], par);)
            if (++it > WAIT_LIMIT) bad = true;
    };
    wait_slot(0, 0);
    wait_slot(1, 0);

    // per-thread geometry
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int ib = i0 + 2 * tx;
    const int jA = j0 + ty, jB = jA + 16;
    const bool inA = ib < nx && jA < ny, inB = ib < nx && jB < ny;
    const bool ylA = jA > 0, yhA = jA < ny - 1, yhB = jB < ny - 1;  // jB > 0 always
    const int oA = (ty + 2) * SBX + 2 * tx + 4, oB = oA + 16 * SBX;  // x-box offsets of (ib, jA/jB)
    const int hA = (ty + 2) * HBX + 2 * tx + 8, hB = hA + 16 * HBX;  // density-box offsets
    // first-colour values are stored compactly, one per two cells of a region
    // row: region column r (0..33) at r / 2. The thread's pair (2tx+1, 2tx+2)
    // holds its first-colour cell at nA + P, P the cell's offset in the pair.
    const int nA = (ty + 1) * NCX + tx, nB = nA + 16 * NCX;
    const size_t plane = (size_t)ny * nx;
    const float h2h = a.h2half;
    const float* __restrict__ fg = a.f;

    // the ring: thread tid < 64 owns side tid/16, position tid%16
    const bool ring = tid < 64;
    const int side = tid >> 4, m = tid & 15;
    auto ring_cell = [&](int q, int& ri, int& rj) {
        if (side < 2) {
            ri = side == 0 ? i0 - 1 : i0 + STX;
            rj = j0 + 2 * m + ((a.c0 + ri + q) & 1);
        } else {
            rj = side == 2 ? j0 - 1 : j0 + STY;
            ri = i0 + 2 * m + ((a.c0 + rj + q) & 1);
        }
    };
    // right sides needed at iteration k: the first colour on plane k+1 and
    // the second colour on plane k (same x), and the ring cell on plane k+1
    auto load_f = [&](int k, float& rA, float& rB, float& bA, float& bB, float& rr) {
        const int q = k + 1;
        const int i = ib + ((a.c0 + jA + q) & 1);
        const float* fq = fg + (size_t)wrapk(q, nz) * plane + i;
        const float* fk = fg + (size_t)wrapk(k, nz) * plane + i;
        rA = inA ? __ldg(fq + (size_t)jA * nx) : 0.f;
        rB = inB ? __ldg(fq + (size_t)jB * nx) : 0.f;
        bA = inA ? __ldg(fk + (size_t)jA * nx) : 0.f;
        bB = inB ? __ldg(fk + (size_t)jB * nx) : 0.f;
        rr = 0.f;
        if (ring) {
            int ri, rj;
            ring_cell(q, ri, rj);
            if (ri >= 0 && ri < nx && rj >= 0 && rj < ny)
                rr = __ldg(fg + (size_t)wrapk(q, nz) * plane + (size_t)rj * nx + ri);
        }
    };
    float fRA, fRB, fBA, fBB, fRR;
    load_f(pbase, fRA, fRB, fBA, fBB, fRR);
    float fPA = 0.f, fPB = 0.f;  // right sides of plane k's first colour (DOT)
    float2 dzf = make_float2(0.f, 0.f), dzq = make_float2(0.f, 0.f);

    // slots of planes k, k+1, k+2 and first-colour planes k-1, k, k+1
    int S1 = 0, S2 = 1, S3 = 2;
    uint32_t par3 = 0;  // parity of slot S3's current fill
    float* N0 = sN + 2 * NPL;
    float* N1 = sN;
    float* N2 = sN + NPL;
    float2 bup1 = make_float2(0.f, 0.f), bup2 = make_float2(0.f, 0.f);  // z+ coefficients, 1 and 2 planes back

    for (int k = pbase; k < k1; ++k) {
        float nRA, nRB, nBA, nBB, nRR;  // next plane's right sides, in flight during this one
        load_f(k + 1, nRA, nRB, nBA, nBB, nRR);
        // DOT: q of this plane's pair, in flight during the first colour
        float2 qa = make_float2(0.f, 0.f), qb = make_float2(0.f, 0.f);
        if (DOT && k >= k0) {
            const float* qo = a.q + (size_t)wrapk(k, nz) * plane + ib;
            if (inA) qa = __ldg(reinterpret_cast<const float2*>(qo + (size_t)jA * nx));
            if (inB) qb = __ldg(reinterpret_cast<const float2*>(qo + (size_t)jB * nx));
        }
        wait_slot(S3, par3);
        const int q = k + 1;
        const int P = (a.c0 + jA + q) & 1;  // x offset of the first colour in the pair on plane q
        const int i = ib + P;
        float2 bdown = make_float2(0.f, 0.f), bup = make_float2(0.f, 0.f);
        // ---- first colour on plane q: the thread's two cells, packed -------
        if (!bad) {
            const __half* Hq = sH + S2 * HPLANE;
            const __half* Hm = sH + S1 * HPLANE;
            const __half* Hp = sH + S3 * HPLANE;
            const float* Xq = sX + S2 * XPLANE;
            const float* Xm = sX + S1 * XPLANE;
            const float* Xp = sX + S3 * XPLANE;
            const int xa = oA + P, xb = oB + P, ha = hA + P, hb = hB + P;
            const float2 rc = make_float2(hval(Hq, ha), hval(Hq, hb));
            float2 num = make_float2(h2h * fRA, h2h * fRB);
            float2 den = make_float2(0.f, 0.f);
            auto acc = [&](float2 b, int dx, const float* X) {
                if (!ZERO) num = __ffma2_rn(b, make_float2(X[xa + dx], X[xb + dx]), num);
                den = __fadd2_rn(den, b);
            };
            // a wall face gets coefficient 0 (no branch: the staged value
            // beyond the wall is the TMA zero fill)
            {
                float2 b = half_beta2(rc, make_float2(hval(Hq, ha - 1), hval(Hq, hb - 1)));
                if (i == 0) b = make_float2(0.f, 0.f);
                acc(b, -1, Xq);
                b = half_beta2(rc, make_float2(hval(Hq, ha + 1), hval(Hq, hb + 1)));
                if (i == nx - 1) b = make_float2(0.f, 0.f);
                acc(b, 1, Xq);
            }
            {
                float2 b = half_beta2(rc, make_float2(hval(Hq, ha - HBX), hval(Hq, hb - HBX)));
                if (!ylA) b.x = 0.f;
                acc(b, -SBX, Xq);
                b = half_beta2(rc, make_float2(hval(Hq, ha + HBX), hval(Hq, hb + HBX)));
                if (!yhA) b.x = 0.f;
                if (!yhB) b.y = 0.f;
                acc(b, SBX, Xq);
            }
            bdown = half_beta2(rc, make_float2(hval(Hm, ha), hval(Hm, hb)));
            acc(bdown, 0, Xm);
            bup = half_beta2(rc, make_float2(hval(Hp, ha), hval(Hp, hb)));
            acc(bup, 0, Xp);
            N2[nA + P] = inA ? __fdividef(num.x, den.x) : 0.f;
            N2[nB + P] = inB ? __fdividef(num.y, den.y) : 0.f;

            if (ring) {  // 16 first-colour ring cells per side (0 outside the domain)
                int ri, rj;
                ring_cell(q, ri, rj);
                float v = 0.f;
                if (ri >= 0 && ri < nx && rj >= 0 && rj < ny) {
                    const int o = (rj - j0 + 2) * SBX + (ri - i0 + 4);
                    const int h = (rj - j0 + 2) * HBX + (ri - i0 + 8);
                    const float r0 = hval(Hq, h);
                    float rn = h2h * fRR, rd = 0.f, b;
                    if (ri > 0) { b = half_beta(r0, hval(Hq, h - 1)); if (!ZERO) rn = fmaf(b, Xq[o - 1], rn); rd += b; }
                    if (ri < nx - 1) { b = half_beta(r0, hval(Hq, h + 1)); if (!ZERO) rn = fmaf(b, Xq[o + 1], rn); rd += b; }
                    if (rj > 0) { b = half_beta(r0, hval(Hq, h - HBX)); if (!ZERO) rn = fmaf(b, Xq[o - SBX], rn); rd += b; }
                    if (rj < ny - 1) { b = half_beta(r0, hval(Hq, h + HBX)); if (!ZERO) rn = fmaf(b, Xq[o + SBX], rn); rd += b; }
                    b = half_beta(r0, hval(Hm, h)); if (!ZERO) rn = fmaf(b, Xm[o], rn); rd += b;
                    b = half_beta(r0, hval(Hp, h)); if (!ZERO) rn = fmaf(b, Xp[o], rn); rd += b;
                    v = __fdividef(rn, rd);
                }
                N2[(rj - j0 + 1) * NCX + ((ri - i0 + 1) >> 1)] = v;
            }
        }
        if (__syncthreads_or(bad)) {
            if (tid == 0) {
                *a.err = 1.0;
                // let the copies already issued land before the block exits
                for (int p = k + 3; p <= issued; ++p) {
                    const int s = (p - pbase) % NSLOT;
                    const uint32_t par = (uint32_t)((p - pbase) / NSLOT) & 1u;
                    for (int it = 0; !mbar_try_wait(&bar[s], par) && it < WAIT_LIMIT; ++it) {
                    }
                }
                if (DOT) a.pa[blin] = a.pb[blin] = 0.0;
            }
            return;
        }
        // ---- second colour on plane k at the same x, written with the first -
        if (k >= k0) {
            const int kk = wrapk(k, nz);
            const __half* Hk = sH + S1 * HPLANE;
            const int ha = hA + P, hb = hB + P, na = nA + P, nb = nB + P;
            const float2 rc = make_float2(hval(Hk, ha), hval(Hk, hb));
            float2 num = make_float2(h2h * fBA, h2h * fBB);
            float2 den = make_float2(0.f, 0.f);
            auto acc = [&](float2 b, float2 xn) {
                num = __ffma2_rn(b, xn, num);
                den = __fadd2_rn(den, b);
            };
            // a wall face gets coefficient 0 (the first-colour value beyond the
            // wall is the ring's 0)
            {
                float2 b = half_beta2(rc, make_float2(hval(Hk, ha - 1), hval(Hk, hb - 1)));
                if (i == 0) b = make_float2(0.f, 0.f);
                acc(b, make_float2(N1[nA], N1[nB]));  // first colour at ib + P - 1
                b = half_beta2(rc, make_float2(hval(Hk, ha + 1), hval(Hk, hb + 1)));
                if (i == nx - 1) b = make_float2(0.f, 0.f);
                acc(b, make_float2(N1[nA + 1], N1[nB + 1]));  // at ib + P + 1
            }
            {
                float2 b = half_beta2(rc, make_float2(hval(Hk, ha - HBX), hval(Hk, hb - HBX)));
                if (!ylA) b.x = 0.f;
                acc(b, make_float2(N1[na - NCX], N1[nb - NCX]));
                b = half_beta2(rc, make_float2(hval(Hk, ha + HBX), hval(Hk, hb + HBX)));
                if (!yhA) b.x = 0.f;
                if (!yhB) b.y = 0.f;
                acc(b, make_float2(N1[na + NCX], N1[nb + NCX]));
            }
            acc(bup2, make_float2(N0[na], N0[nb]));   // face (k-1, k), from the first colour of plane k-1
            acc(bdown, make_float2(N2[na], N2[nb]));  // face (k, k+1), from the first colour of plane k+1
            const float sa = __fdividef(num.x, den.x), sb = __fdividef(num.y, den.y);
            const int pa = nA + (P ^ 1), pb = nB + (P ^ 1);  // first colour of plane k in the pair
            float* xo = a.xout + (size_t)kk * plane + ib;
            const float2 za = P ? make_float2(N1[pa], sa) : make_float2(sa, N1[pa]);
            const float2 zb = P ? make_float2(N1[pb], sb) : make_float2(sb, N1[pb]);
            if (inA) *reinterpret_cast<float2*>(xo + (size_t)jA * nx) = za;
            if (inB) *reinterpret_cast<float2*>(xo + (size_t)jB * nx) = zb;
            if (DOT) {
                if (inA) {
                    dzf = __ffma2_rn(za, P ? make_float2(fPA, fBA) : make_float2(fBA, fPA), dzf);
                    dzq = __ffma2_rn(za, qa, dzq);
                }
                if (inB) {
                    dzf = __ffma2_rn(zb, P ? make_float2(fPB, fBB) : make_float2(fBB, fPB), dzf);
                    dzq = __ffma2_rn(zb, qb, dzq);
                }
            }
        }
        __syncthreads();
        // refill the slot of plane k (no longer read) with plane k + NSLOT
        if (tid == 0 && k + NSLOT <= k1 + 1) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + NSLOT);
        }
        // roll the plane window
        bup2 = bup1;
        bup1 = bup;
        S1 = S2;
        S2 = S3;
        if (++S3 == NSLOT) {
            S3 = 0;
            par3 ^= 1u;  // slot 0 starts its next fill
        }
        float* t = N0;
        N0 = N1;
        N1 = N2;
        N2 = t;
        fPA = fRA;
        fPB = fRB;
        fRA = nRA;
        fRB = nRB;
        fBA = nBA;
        fBB = nBB;
        fRR = nRR;
    }
    if (DOT) {
        const double sf = block_sum((double)dzf.x + (double)dzf.y);
        const double sq = block_sum((double)dzq.x + (double)dzq.y);
        if (tid == 0) {
            a.pa[blin] = sf;
            a.pb[blin] = sq;
        }
    }
}

// Restriction of the residual: the 8 children's residuals summed. The
// fluxes through the 12 faces inside the 2x2x2 block cancel in that sum
// (each leaves one child and enters another), so only the 24 faces on the
// block's boundary are formed:
//   sum_c r_c = sum_c f_c - (1/h^2) sum_{boundary f} beta_f (x_in - x_out).
template <bool B>
__global__ void k_restrict_rho(Bat bt, Dims df, float ih2, const __half* __restrict__ rho,
                               const float* __restrict__ xf, const float* __restrict__ ff, Dims dc,
                               float* __restrict__ fc, int kchunk) {
    const BatBlk bb = bat_blk<B>(bt, blockIdx.z, gridDim.z);
    if (bb.off) return;
    rho = bat_at<B>(bt, bb.cs, rho);
    xf = bat_at<B>(bt, bb.cs, xf);
    ff = bat_at<B>(bt, bb.cs, ff);
    fc = bat_at<B>(bt, bb.cs, fc);
    const int I = blockIdx.x * TBX + threadIdx.x, J = blockIdx.y * TBY + threadIdx.y;
    if (I >= dc.nx || J >= dc.ny) return;
    const int k0 = bb.b * kchunk, k1 = min(k0 + kchunk, dc.nz);
    const int sy = df.nx;
    const bool xl = I > 0, xh = 2 * I + 2 < df.nx, yl = J > 0, yh = 2 * J + 2 < df.ny;
    // the two children of a row (a = 0, 1) are adjacent in x: their x, f and
    // density, and those of their neighbours above, below and across in y,
    // come as pairs (8 and 4 bytes; 2I is even and so is nx)
    auto x2 = [&](int c) { return *reinterpret_cast<const float2*>(xf + c); };
    auto r2 = [&](int c) { return __half22float2(*reinterpret_cast<const __half2*>(rho + c)); };
    for (int K = k0; K < k1; ++K) {
        float fs = 0.f, flux = 0.f;
        const int kk[2] = {2 * K, 2 * K + 1};
        const int kout[2] = {wrapk(2 * K - 1, df.nz), wrapk(2 * K + 2, df.nz)};
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int c = cid(df, 2 * I, 2 * J + b, kk[e]);  // the row's child a = 0
                const int oy = b ? sy : -sy;
                const int cz = cid(df, 2 * I, 2 * J + b, kout[e]);
                const float2 xc = x2(c), rc = r2(c), fc2 = *reinterpret_cast<const float2*>(ff + c);
                const bool hy = b ? yh : yl;
                const float2 xy = hy ? x2(c + oy) : make_float2(0.f, 0.f);
                const float2 ry = hy ? r2(c + oy) : make_float2(0.f, 0.f);
                const float2 xz = x2(cz), rz = r2(cz);
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    // the child's boundary faces: the outer side in x, y and z
                    const float xv = a ? xc.y : xc.x, rv = a ? rc.y : rc.x;
                    fs += a ? fc2.y : fc2.x;
                    const int cx = a ? c + 2 : c - 1;  // its x neighbour outside the block
                    if (a ? xh : xl)
                        flux = fmaf(beta_rho(rv, __half2float(rho[cx])), xv - xf[cx], flux);
                    if (hy)
                        flux = fmaf(beta_rho(rv, a ? ry.y : ry.x), xv - (a ? xy.y : xy.x), flux);
                    flux = fmaf(beta_rho(rv, a ? rz.y : rz.x), xv - (a ? xz.y : xz.x), flux);
                }
            }
        fc[cid(dc, I, J, K)] = 0.125f * (fs - flux * ih2);
    }
}

struct Kahan32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// One block waits, with the sweep's bounded wait, on a shared-memory barrier
// that nothing completes (no copy is issued): the limit runs out and the
// block sets the error flag, as the sweep does when a staged plane never
// arrives (the diagnostic behind vof_diag_wait_timeout).
__global__ void k_wait_probe(double* __restrict__ err, int limit) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool bad = false;
    for (int it = 0; !bad && !mbar_try_wait(&bar, 0u);)
        if (++it > limit) bad = true;
    if (__syncthreads_or(bad) && threadIdx.x == 0) *err = 1.0;
}

// q = A p on the FP32 density with the block partials of p.q, on x-pairs:
// a thread owns cells (2t, 2t+1) of its row and walks up its z chunk
// carrying the pair's plane below and the coefficient of the face below; p
// and the density of the pair, of the pairs across in y and of the pair
// above come as 8-byte loads, the two outer x neighbours as scalars. Each
// cell's stencil is summed over its faces -x, +x, -y, +y, -z, +z; the
// thread's partial of p.q takes the pair's two cells in turn.
template <bool B>
__global__ void k_apply_A_dot_rho32_pair(Bat bt, Dims d, float ih2, const float* __restrict__ rho,
                                         const float* __restrict__ p, float* __restrict__ q,
                                         double* __restrict__ part, int kchunk) {
    const BatBlk bb = bat_blk<B>(bt, blockIdx.z, gridDim.z);
    if (bb.off) return;
    rho = bat_at<B>(bt, bb.cs, rho);
    p = bat_at<B>(bt, bb.cs, p);
    q = bat_at<B>(bt, bb.cs, q);
    part = bat_at<B>(bt, bb.cs, part);
    const int t = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const int i = 2 * t;
    const bool act = i < d.nx && j < d.ny;
    const int k0 = bb.b * kchunk, k1 = min(k0 + kchunk, d.nz);
    Kahan32 ks;
    if (act && k0 < k1) {
        auto ld2 = [](const float* a, int c) { return *reinterpret_cast<const float2*>(a + c); };
        const bool hw = i > 0, he = i + 2 < d.nx, hs = j > 0, hn = j + 1 < d.ny;
        int c = cid(d, i, j, k0);
        const int cb0 = cid(d, i, j, wrapk(k0 - 1, d.nz));
        float2 rc = ld2(rho, c), pc = ld2(p, c);
        const float2 rb = ld2(rho, cb0), pb = ld2(p, cb0);
        float2 bzm = make_float2(beta_rho(rc.x, rb.x), beta_rho(rc.y, rb.y));
        float2 pm = pb;
        for (int k = k0; k < k1; ++k) {
            const int ct = cid(d, i, j, wrapk(k + 1, d.nz));
            const float2 rt = ld2(rho, ct), pt = ld2(p, ct);
            // x: the pair's inner face, and one outer face on either side
            const float rw = hw ? rho[c - 1] : 0.f, pw = hw ? p[c - 1] : 0.f;
            const float re = he ? rho[c + 2] : 0.f, pe = he ? p[c + 2] : 0.f;
            const float bin = beta_rho(rc.x, rc.y);
            const float bxm0 = hw ? beta_rho(rc.x, rw) : 0.f;
            const float bxp1 = he ? beta_rho(rc.y, re) : 0.f;
            const float2 rs = hs ? ld2(rho, c - d.nx) : rc, ps = hs ? ld2(p, c - d.nx) : pc;
            const float2 rn = hn ? ld2(rho, c + d.nx) : rc, pn = hn ? ld2(p, c + d.nx) : pc;
            const float2 bym = hs ? make_float2(beta_rho(rc.x, rs.x), beta_rho(rc.y, rs.y))
                                  : make_float2(0.f, 0.f);
            const float2 byp = hn ? make_float2(beta_rho(rc.x, rn.x), beta_rho(rc.y, rn.y))
                                  : make_float2(0.f, 0.f);
            const float2 bzp = make_float2(beta_rho(rc.x, rt.x), beta_rho(rc.y, rt.y));
            // cell 2t: west neighbour outside the pair, east the pair's other cell
            float s0 = bxm0 * (pc.x - (hw ? pw : pc.x));
            s0 = fmaf(bin, pc.x - pc.y, s0);
            s0 = fmaf(bym.x, pc.x - ps.x, s0);
            s0 = fmaf(byp.x, pc.x - pn.x, s0);
            s0 = fmaf(bzm.x, pc.x - pm.x, s0);
            s0 = fmaf(bzp.x, pc.x - pt.x, s0);
            // cell 2t+1: west the pair's other cell, east neighbour outside
            float s1 = bin * (pc.y - pc.x);
            s1 = fmaf(bxp1, pc.y - (he ? pe : pc.y), s1);
            s1 = fmaf(bym.y, pc.y - ps.y, s1);
            s1 = fmaf(byp.y, pc.y - pn.y, s1);
            s1 = fmaf(bzm.y, pc.y - pm.y, s1);
            s1 = fmaf(bzp.y, pc.y - pt.y, s1);
            const float v0 = s0 * ih2, v1 = s1 * ih2;
            *reinterpret_cast<float2*>(q + c) = make_float2(v0, v1);
            ks.add(pc.x * v0);
            ks.add(pc.y * v1);
            // move up one plane
            bzm = bzp;
            pm = pc;
            rc = rt;
            pc = pt;
            c = ct;
        }
    }
    const double acc = block_sum(ks.value());
    if (threadIdx.x == 0 && threadIdx.y == 0) part[block_linear_z(bb)] = acc;
}

// ---- tensor maps -------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
    });
    return fn;
}

// ncase (nx, ny, nz) arrays of 4- or 2-byte elements, case_stride bytes
// apart (0: a single array), staged in box_x x SBY x 1 boxes, zero outside
bool encode_plane_map(void* store, const Dims& d, const void* base, bool half, int box_x,
                      int ncase = 1, long long case_stride = 0) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const size_t e = half ? sizeof(__half) : sizeof(float);
    const cuuint64_t vol = (cuuint64_t)d.nx * d.ny * d.nz * e;
    const cuuint64_t dims[4] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz,
                                (cuuint64_t)ncase};
    const cuuint64_t strides[3] = {(cuuint64_t)d.nx * e, (cuuint64_t)d.nx * d.ny * e,
                                   ncase > 1 ? (cuuint64_t)case_stride : vol};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)SBY, 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    return fn(reinterpret_cast<CUtensorMap*>(store),
              half ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
              const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool rho_path_eligible(const vof_grid* g, const vof_solver* sv, int nlevels) {
    return sv && sv->precision == VOF_PREC_MIXED_FP32 && sv->mg_interp == VOF_MG_CONSTANT &&
           g->nx % 8 == 0 && nlevels >= 2;  // 16-byte rows of the FP16 density
}

vof_status rho_path_setup(vof_ctx* c) {
    const Level& L0 = c->lv[0];
    if (!encode_plane_map(c->tmap[0], L0.d, L0.xf, false, SBX) ||
        !encode_plane_map(c->tmap[1], L0.d, c->x32b, false, SBX) ||
        !encode_plane_map(c->tmap[2], L0.d, c->rho16, true, HBX))
        return set_err(c, VOF_ERR_CUDA, "TMA tensor-map encoding is unavailable");
    void (*const sweeps[6])(const CUtensorMap, const CUtensorMap, SweepArgs) = {
        k_sweep_rho<true, false, false>, k_sweep_rho<false, false, false>,
        k_sweep_rho<false, true, false>, k_sweep_rho<true, false, true>,
        k_sweep_rho<false, false, true>, k_sweep_rho<false, true, true>};
    bool attr_ok = true;
    for (auto k : sweeps)
        attr_ok = attr_ok && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)SWEEP_SMEM) == cudaSuccess;
    if (!attr_ok)
        return cuda_check(c, cudaGetLastError(), "smoother shared-memory attribute");
    // z chunks: one wave of resident blocks over the whole grid
    const int tiles = ((L0.d.nx + STX - 1) / STX) * ((L0.d.ny + STY - 1) / STY);
    int zc = std::max(1, (SWEEP_BLOCKS_PER_SM * c->sm_count) / tiles);
    zc = std::min(zc, L0.d.nz);
    // at least four planes per block: a block also stages and recomputes
    // two planes below its chunk, which for one plane would triple the work
    // (small grids; the batched ensemble runs many such grids at once)
    c->sweep_kchunk = std::max((L0.d.nz + zc - 1) / zc, std::min(4, L0.d.nz));
    c->sweep_dot = (long)tiles * ((L0.d.nz + c->sweep_kchunk - 1) / c->sweep_kchunk) <= MAX_PARTIALS;
    return VOF_OK;
}

// the TMA maps of a batched solve through case 0's context: every map also
// spans the nc cases, case_stride bytes apart (nc = 1: a single case)
vof_status rho_path_batch_maps(vof_ctx* c, int nc, long long case_stride) {
    const Level& L0 = c->lv[0];
    if (nc > 1 && case_stride % 16 != 0)
        return set_err(c, VOF_ERR_ARG, "batched TMA maps need a 16-byte case stride");
    if (!encode_plane_map(c->tmap[0], L0.d, L0.xf, false, SBX, nc, case_stride) ||
        !encode_plane_map(c->tmap[1], L0.d, c->x32b, false, SBX, nc, case_stride) ||
        !encode_plane_map(c->tmap[2], L0.d, c->rho16, true, HBX, nc, case_stride))
        return set_err(c, VOF_ERR_CUDA, "TMA tensor-map encoding is unavailable");
    return VOF_OK;
}

// one sweep: src == nullptr means the old x is zero; dot: also the dots of
// the new x with the level's right side (slot S_RZ) and with q32 (S_ZQ)
void rho_sweep(vof_ctx* c, const float* src, float* dst, int c0, bool dot) {
    const Level& L0 = c->lv[0];
    SweepArgs a;
    a.nx = L0.d.nx;
    a.ny = L0.d.ny;
    a.nz = L0.d.nz;
    a.h2half = (float)(0.5 * L0.h * L0.h);
    a.c0 = c0;
    a.kchunk = c->sweep_kchunk;
    a.f = L0.ff;
    a.xout = dst;
    a.err = c->scal + S_ERR;
    a.q = c->q32;
    a.pa = c->part + (size_t)S_RZ * MAX_PARTIALS;
    a.pb = c->part + (size_t)S_ZQ * MAX_PARTIALS;
    const CUtensorMap* tx =
        reinterpret_cast<const CUtensorMap*>(src == c->x32b ? c->tmap[1] : c->tmap[0]);
    const CUtensorMap* tr = reinterpret_cast<const CUtensorMap*>(c->tmap[2]);
    const dim3 solo((a.nx + STX - 1) / STX, (a.ny + STY - 1) / STY,
                    (a.nz + a.kchunk - 1) / a.kchunk);
    dim3 grid = solo;
    a.bt = bat_of(c, grid.z);
    int m = timer_begin(c, T_SMOOTH0);
    ++c->nlaunch;
    const bool bat = a.bt.zb != 0;
    auto kern = src == nullptr ? (bat ? k_sweep_rho<true, false, true> : k_sweep_rho<true, false, false>)
                : !dot         ? (bat ? k_sweep_rho<false, false, true> : k_sweep_rho<false, false, false>)
                               : (bat ? k_sweep_rho<false, true, true> : k_sweep_rho<false, true, false>);
    kern<<<grid, dim3(16, 16), SWEEP_SMEM, c->st>>>(*tx, *tr, a);
    timer_end(c, T_SMOOTH0, m);
    if (dot) finalize_dots_beta(c, (int)(solo.x * solo.y * solo.z));
}

void wait_probe(vof_ctx* c, int limit) {
    ++c->nlaunch;
    k_wait_probe<<<1, 32, 0, c->st>>>(c->scal + S_ERR, limit);
}

void rho_restrict(vof_ctx* c) {
    const Level &F = c->lv[0], &C = c->lv[1];
    int m = timer_begin(c, T_RESTRICT0);
    dim3 g = C.L.grid;
    const Bat bt = bat_of(c, g.z);
    auto kern = bt.zb ? k_restrict_rho<true> : k_restrict_rho<false>;
    VOF_LAUNCH(c, kern, g, C.L.block, bt, F.d, (float)(1.0 / (F.h * F.h)),
               (const __half*)c->rho16, F.xf, F.ff, C.d, C.ff, C.L.kchunk);
    timer_end(c, T_RESTRICT0, m);
}

void rho_apply_A_dot(vof_ctx* c, const float* p, float* q, int slot) {
    const Level& L = c->lv[0];
    int m = timer_begin(c, T_RESIDUAL);
    // x-pairs (the density path has nx % 8 == 0): half the blocks across,
    // so twice the z chunks
    const int gx = (L.d.nx / 2 + TBX - 1) / TBX;
    int kchunk = std::max(1, (L.L.kchunk + 1) / 2);
    if ((long)gx * L.L.grid.y * ((L.d.nz + kchunk - 1) / kchunk) > MAX_PARTIALS) kchunk = L.L.kchunk;
    const dim3 solo(gx, L.L.grid.y, (L.d.nz + kchunk - 1) / kchunk);
    dim3 grid = solo;
    const Bat bt = bat_of(c, grid.z);
    auto kern = bt.zb ? k_apply_A_dot_rho32_pair<true> : k_apply_A_dot_rho32_pair<false>;
    VOF_LAUNCH(c, kern, grid, L.L.block, bt, L.d, (float)(1.0 / (L.h * L.h)),
               c->rho32, p, q, c->part + (size_t)slot * MAX_PARTIALS, kchunk);
    timer_end(c, T_RESIDUAL, m);
    finalize_pq_alpha(c, (int)(solo.x * solo.y * solo.z));
}
