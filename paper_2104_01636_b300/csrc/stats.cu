// Running duct statistics on the device (Section 4: profiles averaged over
// the streamwise direction and time, liquid-phase averages alongside the
// mixture ones). For every cross-section column (i, j) the accumulator holds
// FP64 sums over z and over the samples of
//   mixture:          phi = 1 - alpha, u, v, w, uu, vv, ww, uv, uw, vw
//   liquid-weighted:  alpha, alpha u, alpha v, alpha w, alpha uu, alpha vv,
//                     alpha ww, alpha uv, alpha uw, alpha vw
// with the cell-centred velocities. One thread owns a column and sums its z
// planes in order, so the result does not depend on scheduling.
#include <vector>

#include "vof_internal.cuh"

struct vof_stats {
    vof_grid g;
    int dev = 0;
    double* acc = nullptr;  // VOF_NSTAT x ny x nx
    long long samples = 0;
};

namespace {

__global__ void k_stats(Dims d, const double* __restrict__ a, const double* __restrict__ u,
                        const double* __restrict__ v, const double* __restrict__ w,
                        double* __restrict__ acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    double s[VOF_NSTAT];
#pragma unroll
    for (int q = 0; q < VOF_NSTAT; ++q) s[q] = 0.0;
    const size_t plane = (size_t)d.nx * d.ny;
    size_t c = (size_t)j * d.nx + i;
    for (int k = 0; k < d.nz; ++k, c += plane) {
        const double al = a[c], uu = u[c], vv = v[c], ww = w[c];
        const double m[10] = {1.0 - al, uu, vv, ww, uu * uu, vv * vv, ww * ww, uu * vv, uu * ww,
                              vv * ww};
#pragma unroll
        for (int q = 0; q < 10; ++q) s[q] += m[q];
        s[10] += al;
#pragma unroll
        for (int q = 1; q < 10; ++q) s[10 + q] = fma(al, m[q], s[10 + q]);
    }
    const size_t col = (size_t)j * d.nx + i;
#pragma unroll
    for (int q = 0; q < VOF_NSTAT; ++q) acc[q * plane + col] += s[q];
}

}  // namespace

extern "C" {

vof_status vof_stats_create(const vof_grid* grid, vof_stats** out) {
    if (!out || !grid || grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return VOF_ERR_ARG;
    *out = nullptr;
    vof_stats* s = new vof_stats();
    s->g = *grid;
    const size_t bytes = sizeof(double) * VOF_NSTAT * (size_t)grid->nx * grid->ny;
    if (cudaGetDevice(&s->dev) != cudaSuccess || cudaMalloc(&s->acc, bytes) != cudaSuccess ||
        cudaMemset(s->acc, 0, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (s->acc) cudaFree(s->acc);
        delete s;
        return VOF_ERR_OOM;
    }
    *out = s;
    return VOF_OK;
}

vof_status vof_stats_accumulate(vof_stats* s, const double* alpha, const double* uc,
                                const double* vc, const double* wc, void* stream) {
    if (!s || !alpha || !uc || !vc || !wc) return VOF_ERR_ARG;
    const Dims d{s->g.nx, s->g.ny, s->g.nz};
    const dim3 grid((d.nx + 127) / 128, d.ny);
    k_stats<<<grid, 128, 0, (cudaStream_t)stream>>>(d, alpha, uc, vc, wc, s->acc);
    if (cudaGetLastError() != cudaSuccess) return VOF_ERR_CUDA;
    ++s->samples;
    return VOF_OK;
}

vof_status vof_stats_read(vof_stats* s, double* sums, long long* samples) {
    if (!s || !sums || !samples) return VOF_ERR_ARG;
    const size_t bytes = sizeof(double) * VOF_NSTAT * (size_t)s->g.nx * s->g.ny;
    // the accumulations ran on the callers' streams: let them finish
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(sums, s->acc, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    *samples = s->samples;
    return VOF_OK;
}

vof_status vof_stats_reset(vof_stats* s) {
    if (!s) return VOF_ERR_ARG;
    const size_t bytes = sizeof(double) * VOF_NSTAT * (size_t)s->g.nx * s->g.ny;
    if (cudaMemset(s->acc, 0, bytes) != cudaSuccess) return VOF_ERR_CUDA;
    s->samples = 0;
    return VOF_OK;
}

vof_status vof_stats_destroy(vof_stats* s) {
    if (!s) return VOF_ERR_ARG;
    cudaFree(s->acc);
    delete s;
    return VOF_OK;
}

}  // extern "C"
