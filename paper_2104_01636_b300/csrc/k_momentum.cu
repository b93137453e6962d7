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
    const double *u, *v, *w;  // face velocities that advected alpha
    const double *fx, *fy, *fz;
    double rl, rg, ml, mg, rho0, gz, dpdz, dt, h;
    int upwind;
};

__device__ __forceinline__ double vcell(const Pred& P, int comp, int i, int j, int k) {
    double s = 1.0;
    if (i < 0) { i = 0; s = -s; } else if (i >= P.d.nx) { i = P.d.nx - 1; s = -s; }
    if (j < 0) { j = 0; s = -s; } else if (j >= P.d.ny) { j = P.d.ny - 1; s = -s; }
    return s * P.U[comp][cid(P.d, i, j, wrapk(k, P.d.nz))];
}

__device__ __forceinline__ double mucell(const Pred& P, int i, int j, int k) {
    i = min(max(i, 0), P.d.nx - 1);
    j = min(max(j, 0), P.d.ny - 1);
    const double al = P.an[cid(P.d, i, j, wrapk(k, P.d.nz))];
    return al * P.ml + (1.0 - al) * P.mg;
}

__global__ void k_predict(Pred P, double* __restrict__ o0, double* __restrict__ o1,
                          double* __restrict__ o2, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    const Dims& d = P.d;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    const double dt_h = P.dt / P.h;
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        const double rn = P.an[c] * P.rl + (1.0 - P.an[c]) * P.rg;
        const double rn1 = P.a1[c] * P.rl + (1.0 - P.a1[c]) * P.rg;
        const double muc = mucell(P, i, j, k);
        // mass flux and neighbour of each of the six faces (walls: M = 0)
        double M[6];
        int nbc[6];
        double upwL[6];  // 1 if the face's left cell is the donor
        double sgn[6];
        for (int f = 0; f < 6; ++f) {
            const int dd = f >> 1, side = f & 1;
            sgn[f] = side ? 1.0 : -1.0;
            int fi = i, fj = j, fk = k;  // face index in its direction's layout
            bool wall = false;
            double uf = 0.0, F = 0.0;
            if (dd == 0) {
                fi = i + side;
                wall = fi == 0 || fi == d.nx;
                if (!wall) { uf = P.u[uid(d, fi, j, k)]; F = P.fx[uid(d, fi, j, k)]; }
                nbc[f] = side ? (i + 1 < d.nx ? c + 1 : c) : (i > 0 ? c - 1 : c);
            } else if (dd == 1) {
                fj = j + side;
                wall = fj == 0 || fj == d.ny;
                if (!wall) { uf = P.v[vid(d, i, fj, k)]; F = P.fy[vid(d, i, fj, k)]; }
                nbc[f] = side ? (j + 1 < d.ny ? c + d.nx : c) : (j > 0 ? c - d.nx : c);
            } else {
                fk = wrapk(k + side, d.nz);
                uf = P.w[wid(d, i, j, fk)];
                F = P.fz[wid(d, i, j, fk)];
                nbc[f] = cid(d, i, j, wrapk(k + (side ? 1 : -1), d.nz));
            }
            M[f] = wall ? 0.0 : P.rl * F + P.rg * (uf * dt_h - F);
            upwL[f] = uf > 0.0 ? 1.0 : 0.0;
        }
        double out[3];
        for (int comp = 0; comp < 3; ++comp) {
            const double qc = P.U[comp][c];
            // convection
            double C = 0.0;
            for (int f = 0; f < 6; ++f) {
                if (M[f] == 0.0) continue;
                const double qn = P.U[comp][nbc[f]];
                const double qL = (f & 1) ? qc : qn, qR = (f & 1) ? qn : qc;
                const double qs = P.upwind ? (upwL[f] > 0.0 ? qL : qR) : 0.5 * (qL + qR);
                C += sgn[f] * M[f] * qs;
            }
            // viscous traction over the six faces
            double V = 0.0;
            for (int f = 0; f < 6; ++f) {
                const int dd = f >> 1;
                int o[3] = {0, 0, 0};
                o[dd] = (f & 1) ? 1 : -1;
                const int ni = i + o[0], nj = j + o[1], nk = k + o[2];
                const double muf = 0.5 * (muc + mucell(P, ni, nj, nk));
                const double dq = sgn[f] * (vcell(P, comp, ni, nj, nk) - qc) / P.h;
                double tr = dq;
                if (dd != comp) {
                    int e[3] = {0, 0, 0};
                    e[comp] = 1;
                    const double g1 = vcell(P, dd, i + e[0], j + e[1], k + e[2]) -
                                      vcell(P, dd, i - e[0], j - e[1], k - e[2]);
                    const double g2 = vcell(P, dd, ni + e[0], nj + e[1], nk + e[2]) -
                                      vcell(P, dd, ni - e[0], nj - e[1], nk - e[2]);
                    tr = 0.25 * (g1 + g2) / P.h;
                }
                V += sgn[f] * muf * (dq + tr);
            }
            V /= P.h;
            const double B = comp == 2 ? (rn - P.rho0) * P.gz + P.dpdz : 0.0;
            out[comp] = (rn * qc - C + P.dt * (V + B)) / rn1;
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
    VOF_LAUNCH(c, k_predict, L.grid, L.block, P, out[0], out[1], out[2], L.kchunk);
    timer_end(c, T_PREDICT, m);
}

void launch_cell_to_face(vof_ctx* c, const double* uc, const double* vc, const double* wc,
                         double* u, double* v, double* w) {
    const Launch& L = c->Lc;
    int m = timer_begin(c, T_PREDICT);
    VOF_LAUNCH(c, k_cell_to_face, L.grid, L.block, c->d, uc, vc, wc, u, v, w, L.kchunk);
    timer_end(c, T_PREDICT, m);
}
