// Launch geometry and the deterministic second pass of every reduction.
#include "vof_internal.cuh"

Launch launch_cells(int nx, int ny, int nz, int sm_count) {
    Launch L;
    const int gx = (nx + TBX - 1) / TBX, gy = (ny + TBY - 1) / TBY;
    const int target = sm_count * 8;
    int gz = target / (gx * gy);
    if (gz < 1) gz = 1;
    if (gz > nz) gz = nz;
    while (gx * gy * gz > MAX_PARTIALS && gz > 1) --gz;
    L.kchunk = (nz + gz - 1) / gz;
    gz = (nz + L.kchunk - 1) / L.kchunk;
    L.grid = dim3(gx, gy, gz);
    L.block = dim3(TBX, TBY, 1);
    L.nblocks = gx * gy * gz;
    return L;
}

__global__ void k_finalize_sum(const double* __restrict__ part, int n, double* out, double scale) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s * scale;
}

__global__ void k_finalize_max(const double* __restrict__ part, int n, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, part[i]);
    s = block_max(s);
    if (threadIdx.x == 0) *out = s;
}

void finalize_sum(vof_ctx* c, int slot, int nparts, int dst, double scale) {
    VOF_LAUNCH(c, k_finalize_sum, 1, 1024, c->part + (size_t)slot * MAX_PARTIALS, nparts,
                                          c->scal + dst, scale);
}

void finalize_max(vof_ctx* c, int slot, int nparts, int dst) {
    VOF_LAUNCH(c, k_finalize_max, 1, 1024, c->part + (size_t)slot * MAX_PARTIALS, nparts,
                                          c->scal + dst);
}
