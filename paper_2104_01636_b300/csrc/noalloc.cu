// y = A x for the pressure operator without any device allocation.
//
// vof_apply_operator needs a context, and a context allocates its workspace
// with cudaMalloc. This variant is for callers that cannot allocate device
// memory: code running while its stream is being captured into a CUDA graph,
// hosts that reserve all device memory up front through their own arena, and
// latency-critical loops where a cudaMalloc could synchronise the device. The
// scratch it needs -- the face coefficients beta built from alpha -- lives in
// one fixed file-scope device array instead.
#include <mutex>

#include "vof_internal.cuh"

// Face coefficients of one call (x, then y, then z faces), shared by all calls.
static __device__ __align__(256) double g_noalloc_beta[VOF_NOALLOC_MAX_FACES];

namespace {

std::mutex g_mu;
double* g_addr[256] = {nullptr};  // device address of g_noalloc_beta per device ordinal

__global__ void k_na_beta(Dims d, const double* __restrict__ a, double rl, double rg,
                          double* __restrict__ bx, double* __restrict__ by,
                          double* __restrict__ bz, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
        const int c = cid(d, i, j, k);
        const double rc = a[c] * rl + (1.0 - a[c]) * rg;
        if (i == 0) {
            bx[uid(d, 0, j, k)] = 0.0;
        } else {
            const double rw = a[c - 1] * rl + (1.0 - a[c - 1]) * rg;
            bx[uid(d, i, j, k)] = 1.0 / (0.5 * (rw + rc));
        }
        if (i == d.nx - 1) bx[uid(d, d.nx, j, k)] = 0.0;
        if (j == 0) {
            by[vid(d, i, 0, k)] = 0.0;
        } else {
            const double rs = a[c - d.nx] * rl + (1.0 - a[c - d.nx]) * rg;
            by[vid(d, i, j, k)] = 1.0 / (0.5 * (rs + rc));
        }
        if (j == d.ny - 1) by[vid(d, i, d.ny, k)] = 0.0;
        const int cb = cid(d, i, j, wrapk(k - 1, d.nz));
        const double rb = a[cb] * rl + (1.0 - a[cb]) * rg;
        bz[wid(d, i, j, k)] = 1.0 / (0.5 * (rb + rc));
    }
}

__global__ void k_na_apply(Dims d, double ih2, const double* __restrict__ bx,
                           const double* __restrict__ by, const double* __restrict__ bz,
                           const double* __restrict__ x, double* __restrict__ y, int kchunk) {
    const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int k0 = blockIdx.z * kchunk, k1 = min(k0 + kchunk, d.nz);
    for (int k = k0; k < k1; ++k) {
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
        y[c] = s * ih2;
    }
}

// Device address of the scratch on the current device, looked up once per
// device (cudaGetSymbolAddress may load the module, so this first lookup
// must not happen inside a stream capture).
vof_status scratch_on_current_device(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_beta) != cudaSuccess || !p) {
            cudaGetLastError();
            return VOF_ERR_CUDA;
        }
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return VOF_OK;
}

}  // namespace

extern "C" vof_status vof_apply_operator_noalloc(const vof_grid* grid, const vof_phys* phys,
                                                 const double* alpha, const double* x, double* y,
                                                 void* stream) {
    if (!grid || !phys || !alpha || !x || !y) return VOF_ERR_ARG;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || !(grid->h > 0.0)) return VOF_ERR_ARG;
    if (grid->periodic_x || grid->periodic_y) return VOF_ERR_UNSUPPORTED;
    if (!(phys->rho_l > 0.0) || !(phys->rho_g > 0.0)) return VOF_ERR_ARG;
    const size_t nu = (size_t)(grid->nx + 1) * grid->ny * grid->nz;
    const size_t nv = (size_t)grid->nx * (grid->ny + 1) * grid->nz;
    const size_t nw = (size_t)grid->nx * grid->ny * grid->nz;
    if (nu + nv + nw > (size_t)VOF_NOALLOC_MAX_FACES) return VOF_ERR_ADMISSION;
    const long tiles = (long)((grid->nx + TBX - 1) / TBX) * ((grid->ny + TBY - 1) / TBY);
    if (tiles > MAX_PARTIALS) return VOF_ERR_ARG;
    double* beta = nullptr;
    vof_status st = scratch_on_current_device(&beta);
    if (st != VOF_OK) return st;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    const Dims d{grid->nx, grid->ny, grid->nz};
    const Launch L = launch_cells(d.nx, d.ny, d.nz, sms);
    cudaStream_t s = (cudaStream_t)stream;
    double* bx = beta;
    double* by = beta + nu;
    double* bz = beta + nu + nv;
    k_na_beta<<<L.grid, L.block, 0, s>>>(d, alpha, phys->rho_l, phys->rho_g, bx, by, bz, L.kchunk);
    k_na_apply<<<L.grid, L.block, 0, s>>>(d, 1.0 / (grid->h * grid->h), bx, by, bz, x, y,
                                          L.kchunk);
    if (cudaGetLastError() != cudaSuccess) return VOF_ERR_CUDA;
    return VOF_OK;
}
