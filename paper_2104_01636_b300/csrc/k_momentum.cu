// Momentum predictor (Eq. 2; Section 2.2 steps 8-10) on the collocated grid:
// the momentum variable is the cell-centred velocity, convected with the
// mass fluxes of the geometric VOF sweep,
//   M_f = rho_l F_f + rho_g (u_f dt/h - F_f),
// F_f the liquid volume the sweep moved through face f (cell volumes), so
// that rho^{n+1} from alpha^{n+1} is the density these same fluxes produce:
//   rho^{n+1} u_hat = rho^n u^n - sum_f (+-) M_f q*_f + dt (V + B),
// with q*_f the donor cell's velocity (upwind) or the two-cell mean
// (central), V the explicit full-stress viscous force (face viscosity the
// linear average of the two cells, step 10; tangential derivatives averaged
// from the central differences in both cells) and on the z-component
// B = (rho^n - rho0) g_z + dpdz (Section 4). Walls: no-slip ghosts (every
// velocity component changes sign), mirrored viscosity, no mass flux.
// Step 10: face velocities u_hat_f = mean of the two cells.
#include "vof_internal.cuh"

namespace {

struct Pred {
    Dims d;
    const double *an, *a1;    // alpha^n, alpha^{n+1}
    const double* U[3];       // cell velocities at level n
    const float* U32[3];      // their FP32 copies (mixed path: viscous term)
    const float* a32;         // alpha^n in FP32 (mixed path: face viscosities)
    const double *u, *v, *w;  // face velocities that advected alpha
    const double *fx, *fy, *fz;
    double rl, rg, ml, mg, rho0, gz, dpdz, dt, h;
    int upwind;
};

// velocity component with no-slip ghosts: every component changes sign
// across a wall (the sign is applied as a negation, not a multiply)
template <class VT>
__device__ __forceinline__ VT vcell(const Pred& P, const VT* const* U, int comp, int i, int j,
                                    int k) {
    bool flip = false;
    if (i < 0) { i = 0; flip = !flip; } else if (i >= P.d.nx) { i = P.d.nx - 1; flip = !flip; }
    if (j < 0) { j = 0; flip = !flip; } else if (j >= P.d.ny) { j = P.d.ny - 1; flip = !flip; }
    const VT q = U[comp][cid(P.d, i, j, wrapk(k, P.d.nz))];
    return flip ? -q : q;
}

template <class VT> __device__ __forceinline__ const VT* const* visc_src(const Pred& P);
template <> __device__ __forceinline__ const double* const* visc_src<double>(const Pred& P) {
    return P.U;
}
template <> __device__ __forceinline__ const float* const* visc_src<float>(const Pred& P) {
    return P.U32;
}

// 1 / s without a division: an FP32 reciprocal seed r (relative error e0
// below 2^-22) refined by one third-order step r + r (e + e^2), e = 1 - s r,
// whose truncation error e0^3 < 2^-66 lies below FP64 rounding; s is a
// density, a normal positive number
__device__ __forceinline__ double rcp_cubic(double s) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"((float)s));
    const double r = (double)r0;
    const double e = fma(-s, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// mu of a cell from its volume fraction, in the viscous term's precision
template <class VT> __device__ __forceinline__ VT mu_cell(const Pred& P, int c);
template <> __device__ __forceinline__ double mu_cell<double>(const Pred& P, int c) {
    return fma(P.an[c], P.ml - P.mg, P.mg);
}
template <> __device__ __forceinline__ float mu_cell<float>(const Pred& P, int c) {
    return fmaf(P.a32[c], (float)(P.ml - P.mg), (float)P.mg);
}

// VT: arithmetic of the viscous term (double on the FP64 path; float on the
// mixed path, where it changes the velocity by ~1e-4 of itself per step).
// The mass fluxes, densities, body force and the update are FP64 on both
// paths; the face viscosities are formed in VT. On the mixed path the
// convective and viscous increments are combined in FP32 before the FP64
// update, and the net outward flux is summed in FP32 from the rounded
// fluxes. On the mixed path the transport sum
// sum_f M_f q*_f is also taken in FP32 (fluxes rounded once, FP32 copies of the
// cell velocities): it is rounded to 6e-8 of the convective change, which is a
// fraction of the velocity, so u_hat moves by ~1e-8 of itself. Central
// convection uses sum_f (+-) M_f (q_c + q_nb)/2 = (q_c net + sum_f (+-) M_f
// q_nb)/2 with the net outward mass flux formed once per cell; each
// tangential derivative at the cell is formed once and shared by its two
// faces. The mixed variant is held to 128 registers: two blocks per SM.
template <class VT>
__global__ void __launch_bounds__(TBX * TBY, sizeof(VT) == sizeof(float) ? 2 : 1)
    k_predict(Pred P, double* __restrict__ o0, double* __restrict__ o1, double* __restrict__ o2,
              int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const Dims& d = P.d;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    const double inv_h = 1.0 / P.h;
    const VT dt_ih2 = (VT)(P.dt * inv_h * inv_h);  // dt / h^2, the viscous term's scale
    const double drho = P.rl - P.rg;
    // half mass fluxes M / 2 (exact halving: the central average's 1/2 is
    // folded into them)
    const double drho_h = 0.5 * drho;
    const double rg_dth_h = 0.5 * P.rg * (P.dt * inv_h);
    // dt B on z: dt ((rho^n - rho0) g_z + dpdz) = rho^n (dt g_z) + dt (dpdz - rho0 g_z)
    const double dt_gz = P.dt * P.gz, dt_b0 = P.dt * (P.dpdz - P.rho0 * P.gz);
    const VT* const* UV = visc_src<VT>(P);
    constexpr bool MIXED = sizeof(VT) == sizeof(float);
    // the -z face of plane k is the +z face of plane k - 1: its half flux and
    // face velocity carry over along the march (the same expression, formed
    // once); planes k0's -z face is formed at the start
    double M_up = 0.0, uf_up = 0.0;
    {
        const int fk = wrapk(k0, d.nz);
        uf_up = P.w[wid(d, i, j, fk)];
        M_up = fma(drho_h, P.fz[wid(d, i, j, fk)], rg_dth_h * uf_up);
    }
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        const double an = P.an[c];
        const double rn = fma(an, drho, P.rg);
        const double rn1 = fma(P.a1[c], drho, P.rg);
        const VT muc = mu_cell<VT>(P, c);
        // per face f (0,1: -x,+x; 2,3: -y,+y; 4,5: -z,+z): neighbour cell
        // (clamped at walls), face viscosity, signed outward mass flux (0 on
        // walls), donor side
        int nbc[6];
        VT muf[6];
        double Ms[6];  // outward-signed half fluxes: -M/2 on minus faces, +M/2 on plus faces
        bool left_donor[6];
        double net = 0.0;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int dd = f >> 1, side = f & 1;
            int ni = i, nj = j, nk = k;
            bool wall = false;
            double uf = 0.0, F = 0.0;
            if (dd == 0) {
                ni = side ? i + 1 : i - 1;
                const int fi = i + side;
                wall = fi == 0 || fi == d.nx;
                if (!wall) { uf = P.u[uid(d, fi, j, k)]; F = P.fx[uid(d, fi, j, k)]; }
            } else if (dd == 1) {
                nj = side ? j + 1 : j - 1;
                const int fj = j + side;
                wall = fj == 0 || fj == d.ny;
                if (!wall) { uf = P.v[vid(d, i, fj, k)]; F = P.fy[vid(d, i, fj, k)]; }
            } else {
                nk = side ? k + 1 : k - 1;
                if (side) {
                    const int fk = wrapk(k + 1, d.nz);
                    uf = P.w[wid(d, i, j, fk)];
                    F = P.fz[wid(d, i, j, fk)];
                } else {
                    uf = uf_up;
                }
            }
            const int ci = min(max(ni, 0), d.nx - 1), cj = min(max(nj, 0), d.ny - 1);
            nbc[f] = cid(d, ci, cj, wrapk(nk, d.nz));
            muf[f] = VT(0.5) * (muc + mu_cell<VT>(P, nbc[f]));
            const double M = f == 4 ? M_up : (wall ? 0.0 : fma(drho_h, F, rg_dth_h * uf));
            if (f == 5) {
                M_up = M;
                uf_up = uf;
            }
            Ms[f] = side ? M : -M;
            if constexpr (!MIXED) net += Ms[f];
            // u_f > 0 as a sign test of the bits (no FP64 compare; +-0 is not > 0)
            left_donor[f] = __double_as_longlong(uf) > 0LL;
        }
        const double r_rn1 = rcp_cubic(rn1);
        float Msf[6];
        float netf = 0.f;
        if constexpr (MIXED) {
            // the net outward flux summed in FP32 from the rounded fluxes
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                Msf[f] = (float)Ms[f];
                netf += Msf[f];
            }
        }
        double out[3];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp) {
            const double qc = P.U[comp][c];
            // convection: outward mass flux times the transported velocity
            double C = 0.0;
            float Cm = 0.f;  // the mixed path's FP32 sum
            if constexpr (sizeof(VT) == sizeof(float)) {
                // mixed path: the transport sum in FP32 from the FP32 copies
                const float* Q = P.U32[comp];
                const float qcf = Q[c];
                float Cf = 0.f;
                if (P.upwind) {
#pragma unroll
                    for (int f = 0; f < 6; ++f) {
                        const bool own = (f & 1) ? left_donor[f] : !left_donor[f];
                        Cf = fmaf(Msf[f], own ? qcf : Q[nbc[f]], Cf);
                    }
                    Cf = 2.f * Cf;
                } else {
                    float sf = 0.f;
#pragma unroll
                    for (int f = 0; f < 6; ++f) sf = fmaf(Msf[f], Q[nbc[f]], sf);
                    Cf = fmaf(netf, qcf, sf);
                }
                Cm = Cf;
            } else if (P.upwind) {
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                    const double qn = P.U[comp][nbc[f]];
                    // donor: the left cell when u_f > 0 (plus face: this cell)
                    const bool own = (f & 1) ? left_donor[f] : !left_donor[f];
                    C = fma(Ms[f], own ? qc : qn, C);
                }
                C = 2.0 * C;
            } else {
                double s = 0.0;
#pragma unroll
                for (int f = 0; f < 6; ++f) s = fma(Ms[f], P.U[comp][nbc[f]], s);
                C = fma(net, qc, s);
            }
            // viscous: (1/h^2) sum_f mu_f [(q_nb - q_c) + s_f (tangential difference)/4]
            const VT qcv = UV[comp][c];
            VT g1[3];  // central difference of component dd along comp at the cell
#pragma unroll
            for (int dd = 0; dd < 3; ++dd) {
                if (dd == comp) { g1[dd] = VT(0); continue; }
                int e[3] = {0, 0, 0};
                e[comp] = 1;
                g1[dd] = vcell<VT>(P, UV, dd, i + e[0], j + e[1], k + e[2]) -
                         vcell<VT>(P, UV, dd, i - e[0], j - e[1], k - e[2]);
            }
            VT V = VT(0);
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const int dd = f >> 1;
                int o[3] = {0, 0, 0};
                o[dd] = (f & 1) ? 1 : -1;
                const int ni = i + o[0], nj = j + o[1], nk = k + o[2];
                const VT diff = vcell<VT>(P, UV, comp, ni, nj, nk) - qcv;
                VT t;
                if (dd == comp) {
                    t = diff + diff;
                } else {
                    int e[3] = {0, 0, 0};
                    e[comp] = 1;
                    const VT g2 = vcell<VT>(P, UV, dd, ni + e[0], nj + e[1], nk + e[2]) -
                                  vcell<VT>(P, UV, dd, ni - e[0], nj - e[1], nk - e[2]);
                    t = fma((f & 1) ? VT(0.25) : VT(-0.25), g1[dd] + g2, diff);
                }
                V = fma(muf[f], t, V);
            }
            // rho^n q - C + dt (V / h^2 + B), B on z only
            if constexpr (MIXED) {
                // convection and viscous term combined in FP32 (each a fraction
                // of the momentum); the body force stays FP64: in the liquid
                // rho^n dt g_z and dt (dpdz - rho0 g_z) nearly cancel
                double num = fma(rn, qc, (double)fmaf(V, dt_ih2, -Cm));
                if (comp == 2) num += fma(rn, dt_gz, dt_b0);
                out[comp] = num * r_rn1;
            } else {
                double num = fma(rn, qc, -C) + (double)(V * dt_ih2);
                if (comp == 2) num += fma(rn, dt_gz, dt_b0);
                out[comp] = num * r_rn1;
            }
        }
        o0[c] = out[0];
        o1[c] = out[1];
        o2[c] = out[2];
    }
}

// step 10: face value = mean of the two cells (zero on walls)
__global__ void k_cell_to_face(Dims d, const double* __restrict__ uc, const double* __restrict__ vc,
                               const double* __restrict__ wc, double* __restrict__ u,
                               double* __restrict__ v, double* __restrict__ w, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        u[uid(d, i, j, k)] = i == 0 ? 0.0 : 0.5 * (uc[c - 1] + uc[c]);
        if (i == d.nx - 1) u[uid(d, d.nx, j, k)] = 0.0;
        v[vid(d, i, j, k)] = j == 0 ? 0.0 : 0.5 * (vc[c - d.nx] + vc[c]);
        if (j == d.ny - 1) v[vid(d, i, d.ny, k)] = 0.0;
        w[wid(d, i, j, k)] = 0.5 * (wc[cid(d, i, j, wrapk(k - 1, d.nz))] + wc[c]);
    }
}

}  // namespace

void launch_predict(vof_ctx* c, const double* alpha_n, const double* alpha_np1,
                    const double* const U[3], const double* u, const double* v, const double* w,
                    const double* fx, const double* fy, const double* fz, double dt,
                    double* const out[3]) {
    const Launch& L = c->Lc;
    Pred P;
    P.d = c->d;
    P.an = alpha_n;
    P.a1 = alpha_np1;
    for (int q = 0; q < 3; ++q) P.U[q] = U[q];
    P.u = u;
    P.v = v;
    P.w = w;
    P.fx = fx;
    P.fy = fy;
    P.fz = fz;
    P.rl = c->ph.rho_l;
    P.rg = c->ph.rho_g;
    P.ml = c->ph.mu_l;
    P.mg = c->ph.mu_g;
    P.rho0 = c->ph.rho0;
    P.gz = c->ph.g_z;
    P.dpdz = c->ph.dpdz;
    P.dt = dt;
    P.h = c->g.h;
    P.upwind = c->ph.conv_scheme == VOF_CONV_UPWIND;
    int m = timer_begin(c, T_PREDICT);
    if (c->sv.precision == VOF_PREC_MIXED_FP32) {
        // FP32 copies of the cell velocities and of alpha^n for the viscous term
        const int n = c->d.nx * c->d.ny * c->d.nz;
        for (int q = 0; q < 3; ++q) {
            mg_to_f32(c, U[q], c->u32[q], n);
            P.U32[q] = c->u32[q];
        }
        mg_to_f32(c, alpha_n, c->u32[3], n);
        P.a32 = c->u32[3];
        VOF_LAUNCH(c, k_predict<float>, L.grid, L.block, P, out[0], out[1], out[2], L.kchunk);
    } else {
        for (int q = 0; q < 3; ++q) P.U32[q] = nullptr;
        P.a32 = nullptr;
        VOF_LAUNCH(c, k_predict<double>, L.grid, L.block, P, out[0], out[1], out[2], L.kchunk);
    }
    timer_end(c, T_PREDICT, m);
}

void launch_cell_to_face(vof_ctx* c, const double* uc, const double* vc, const double* wc,
                         double* u, double* v, double* w) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_PREDICT);
    VOF_LAUNCH(c, k_cell_to_face, L.grid, L.block, c->d, uc, vc, wc, u, v, w, L.kchunk);
    timer_end(c, T_PREDICT, m);
}
